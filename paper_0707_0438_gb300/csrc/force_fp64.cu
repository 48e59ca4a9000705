// FP64 direct-summation kernel: acceleration, jerk and potential (Sect. 3,
// Sect. 3.1) with every operation in double precision.  It is the accuracy
// reference on the GPU and the baseline the mixed kernel is measured against.
//
// Same staging as the mixed kernel (bulk copies into a shared-memory ring,
// j-groups inside the CTA, j-split over CTAs), one i-particle per thread.  The
// pair j = i is excluded by index, exactly as in the definition; a pair at
// zero separation contributes nothing and s^2 is floored at r_min^2.
// MODE_ACC_POT drops the jerk; MODE_ADJOINT computes dL/dx (jerk slots) and
// dL/dm (potential slot) from g = dL/da held in the velocity slots.
#include <cuda_runtime.h>

#include "kirin_internal.cuh"
#include "tma.cuh"

namespace kirin {
namespace {

__device__ __forceinline__ void write_out64(const ForceArgs &A, int q, int k, double val)
{
    if (k >= A.n_i)
        return;
    if (A.n_split > 1)
        A.partial[((size_t)blockIdx.y * A.nq + q) * A.n_i_pad + k] = val;
    else
        store_final(A, q, k, val);
}

__device__ __forceinline__ void write_nn64(const ForceArgs &A, int k, double r2, double j)
{
    if (k >= A.n_i)
        return;
    if (A.n_split > 1) {
        A.partial[((size_t)blockIdx.y * A.nq + 7) * A.n_i_pad + k] = r2;
        A.partial[((size_t)blockIdx.y * A.nq + 8) * A.n_i_pad + k] = j;
    } else {
        store_nn(A, k, r2, j);
    }
}

// Dynamic shared memory: the tile ring, reused as the [GROUPS][nq][I_CTA]
// doubles of the cross-group reduction after the loop.
constexpr size_t F64_RING_BYTES = (size_t)STAGES * TILE_J * sizeof(JF64);
constexpr size_t F64_RED_BYTES = (size_t)9 * FORCE_THREADS * sizeof(double);
constexpr size_t F64_SMEM_BYTES = F64_RING_BYTES > F64_RED_BYTES ? F64_RING_BYTES : F64_RED_BYTES;

template <int GROUPS, int MODE>
__global__ void __launch_bounds__(FORCE_THREADS) k_force_fp64(const ForceArgs Ain)
{
    ForceArgs A = Ain;
    if (Ain.n_i_dev)
        A.n_i = *Ain.n_i_dev;
    constexpr bool ADJ = MODE == MODE_ADJOINT;
    constexpr bool NN = MODE == MODE_NN;
    constexpr bool JERK = MODE == MODE_ACC_JERK_POT || NN;
    constexpr int NQ = NN ? 9 : 7;
    constexpr int GT = FORCE_THREADS / GROUPS;
    constexpr int I_CTA = GT;
    constexpr int JG = TILE_J / GROUPS;
    constexpr uint32_t TILE_BYTES = TILE_J * sizeof(JF64);
    static_assert(GT >= 32, "a warp must read one j at a time");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    JF64 *tiles = reinterpret_cast<JF64 *>(smem_raw);
    __shared__ __align__(8) uint64_t bars[STAGES];
    if ((long long)blockIdx.x * I_CTA >= A.n_i)
        return;  // beyond the block of a device-driven launch (uniform over the CTA)

    const int tid = threadIdx.x;
    const int g = tid / GT;
    const int s = tid - g * GT;
    const JF64 *__restrict__ J = static_cast<const JF64 *>(A.jimg);

    const int kslot = blockIdx.x * I_CTA + s;
    int i = -1;
    if (kslot < A.n_i) {
        i = A.ilist ? A.ilist[kslot] : kslot;
        if (i < 0 || i >= A.n_j) {
            atomicOr(A.err, ERR_INDEX);
            i = -1;
        }
    }
    const JF64 ri = J[i >= 0 ? i : 0];
    const double xi = ri.q[0].x, yi = ri.q[0].y, zi = ri.q[1].x;
    const double vxi = ri.q[2].x, vyi = ri.q[2].y, vzi = ri.q[3].x;  // g_k in adjoint mode
    const double mk = ri.q[1].y;
    const double eps2 = A.eps2, rmin2 = A.rmin2;

    const int y = blockIdx.y;
    const int tb = A.tile0 + (int)(((long long)A.ntiles * y) / A.n_split);
    const int te = A.tile0 + (int)(((long long)A.ntiles * (y + 1)) / A.n_split);
    const int nt = te - tb;

    if (tid == 0) {
#pragma unroll
        for (int st = 0; st < STAGES; ++st)
            mbar_init(&bars[st], 1);
        mbar_fence_init();
    }
    const uint64_t pol = l2_policy_evict_last();
    __syncthreads();
    if (tid == 0) {
        for (int st = 0; st < STAGES && st < nt; ++st) {
            mbar_arrive_expect_tx(&bars[st], TILE_BYTES);
            bulk_g2s_hint(tiles + st * TILE_J, J + (size_t)(tb + st) * TILE_J, TILE_BYTES, &bars[st], pol);
        }
    }

    double ax = 0, ay = 0, az = 0, jx = 0, jy = 0, jz = 0, pt = 0;
    double nn_r2 = INFINITY;  // nearest j != i so far (strict < in increasing j: smallest index on ties)
    int nn_j = -1;
    int k = 0;
    bool aborted = false;
    for (; k < nt; ++k) {
        const int st = k % STAGES;
        const uint32_t par = (uint32_t)(k / STAGES) & 1u;
        const bool ok = mbar_wait_bounded(&bars[st], par);
        if (ok) {
            const JF64 *__restrict__ T = tiles + st * TILE_J + g * JG;
            const int jbase = (tb + k) * TILE_J + g * JG;
#pragma unroll 2
            for (int jj = 0; jj < JG; ++jj) {
                const double2 p0 = T[jj].q[0], p1 = T[jj].q[1], w0 = T[jj].q[2], w1 = T[jj].q[3];
                const double dx = p0.x - xi, dy = p0.y - yi, dz = p1.x - zi;
                const double wx = w0.x - vxi, wy = w0.y - vyi, wz = w1.x - vzi;
                double s2;
                if (NN) {  // the search compares |d|^2 (padding j >= n_j and j = i skipped)
                    const double d2 = fma(dz, dz, fma(dy, dy, dx * dx));
                    s2 = d2 + eps2;
                    if (jbase + jj != i && jbase + jj < A.n_j && d2 < nn_r2) {
                        nn_r2 = d2;
                        nn_j = jbase + jj;
                    }
                } else {
                    s2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps2)));
                }
                double rinv = rsqrt(fmax(s2, rmin2));
                rinv = (s2 == 0.0 || jbase + jj == i) ? 0.0 : rinv;
                const double rinv2 = rinv * rinv;
                if (ADJ) {
                    // w = m_k g_j - m_j g_k;  dL/dx_k += K(d) w;  dL/dm_k -= g_j.d / s^3
                    const double ri3 = rinv * rinv2;
                    const double ux = mk * w0.x - p1.y * vxi;
                    const double uy = mk * w0.y - p1.y * vyi;
                    const double uz = mk * w1.x - p1.y * vzi;
                    const double du = fma(dz, uz, fma(dy, uy, dx * ux));
                    const double b = 3.0 * du * rinv2 * ri3;
                    jx = fma(ri3, ux, fma(-b, dx, jx));
                    jy = fma(ri3, uy, fma(-b, dy, jy));
                    jz = fma(ri3, uz, fma(-b, dz, jz));
                    pt = fma(fma(w1.x, dz, fma(w0.y, dy, w0.x * dx)), ri3, pt);
                    continue;
                }
                const double mr = p1.y * rinv;
                const double mr3 = mr * rinv2;
                pt += mr;
                ax = fma(mr3, dx, ax);
                ay = fma(mr3, dy, ay);
                az = fma(mr3, dz, az);
                if (JERK) {
                    const double dw = fma(dz, wz, fma(dy, wy, dx * wx));
                    const double b = 3.0 * dw * rinv2 * mr3;
                    jx = fma(mr3, wx, fma(-b, dx, jx));
                    jy = fma(mr3, wy, fma(-b, dy, jy));
                    jz = fma(mr3, wz, fma(-b, dz, jz));
                }
            }
        }
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        if (tid == 0 && k + STAGES < nt) {
            mbar_arrive_expect_tx(&bars[st], TILE_BYTES);
            bulk_g2s_hint(tiles + st * TILE_J, J + (size_t)(tb + k + STAGES) * TILE_J, TILE_BYTES, &bars[st], pol);
        }
    }
    if (aborted) {
        if (tid == 0) {
            const int last = min(nt, k + STAGES);
            for (int kk = k; kk < last; ++kk) {
                if (!mbar_wait_bounded(&bars[kk % STAGES], (uint32_t)(kk / STAGES) & 1u)) {
                    atomicOr(A.err, ERR_DRAIN);
                    break;
                }
            }
            atomicOr(A.err, ERR_TIMEOUT);
        }
        return;
    }
    const double res[7] = {ax, ay, az, jx, jy, jz, pt};
    if (GROUPS == 1) {
#pragma unroll
        for (int q = 0; q < 7; ++q)
            write_out64(A, q, kslot, res[q]);
        if (NN)
            write_nn64(A, kslot, nn_r2, (double)nn_j);
    } else {
        __syncthreads();
        static_assert((size_t)GROUPS * NQ * I_CTA * sizeof(double) <= F64_SMEM_BYTES, "reduction space");
        double *red = reinterpret_cast<double *>(smem_raw);  // [GROUPS][NQ][I_CTA]
#pragma unroll
        for (int q = 0; q < 7; ++q)
            red[(g * NQ + q) * I_CTA + s] = res[q];
        if (NN) {
            red[(g * NQ + 7) * I_CTA + s] = nn_r2;
            red[(g * NQ + 8) * I_CTA + s] = (double)nn_j;
        }
        __syncthreads();
        for (int o = tid; o < 7 * I_CTA; o += FORCE_THREADS) {
            const int q = o / I_CTA;
            const int slot = o - q * I_CTA;
            double sum = 0.0;
#pragma unroll
            for (int gg = 0; gg < GROUPS; ++gg)
                sum += red[(gg * NQ + q) * I_CTA + slot];
            write_out64(A, q, blockIdx.x * I_CTA + slot, sum);
        }
        if (NN) {
            for (int slot = tid; slot < I_CTA; slot += FORCE_THREADS) {
                double r2 = INFINITY, j = -1.0;
#pragma unroll
                for (int gg = 0; gg < GROUPS; ++gg)
                    nn_min(r2, j, red[(gg * NQ + 7) * I_CTA + slot], red[(gg * NQ + 8) * I_CTA + slot]);
                write_nn64(A, blockIdx.x * I_CTA + slot, r2, j);
            }
        }
    }
}

template <int GROUPS, int MODE>
cudaError_t launch_t(const ForceArgs &a, int n_split, cudaStream_t st)
{
    constexpr int I_CTA = FORCE_THREADS / GROUPS;
    const int iblocks = (a.n_i + I_CTA - 1) / I_CTA;
    if (iblocks == 0)
        return cudaSuccess;
    const size_t smem = F64_SMEM_BYTES;
    if (smem > 48 * 1024) {
        static bool opted = false;  // per template instance
        if (!opted) {
            cudaFuncSetAttribute(k_force_fp64<GROUPS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            opted = true;
        }
    }
    dim3 grid(iblocks, n_split);
    k_force_fp64<GROUPS, MODE><<<grid, FORCE_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

template <int GROUPS, int MODE>
int occ_t()
{
    int n = 0;
    const size_t smem = F64_SMEM_BYTES;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_force_fp64<GROUPS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_force_fp64<GROUPS, MODE>, FORCE_THREADS, smem);
    return n;
}

template <int MODE>
cudaError_t launch_g(const ForceArgs &a, Shape s, cudaStream_t st)
{
    switch (s.groups) {
    case 1: return launch_t<1, MODE>(a, s.n_split, st);
    case 2: return launch_t<2, MODE>(a, s.n_split, st);
    case 4: return launch_t<4, MODE>(a, s.n_split, st);
    case 8: return launch_t<8, MODE>(a, s.n_split, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int MODE>
int occ_g(int groups)
{
    switch (groups) {
    case 1: return occ_t<1, MODE>();
    case 2: return occ_t<2, MODE>();
    case 4: return occ_t<4, MODE>();
    case 8: return occ_t<8, MODE>();
    default: return 0;
    }
}

}  // namespace

cudaError_t launch_force_fp64(const ForceArgs &a, Shape s, int mode, cudaStream_t st)
{
    switch (mode) {
    case MODE_ACC_JERK_POT: return launch_g<MODE_ACC_JERK_POT>(a, s, st);
    case MODE_ACC_POT: return launch_g<MODE_ACC_POT>(a, s, st);
    case MODE_ADJOINT: return launch_g<MODE_ADJOINT>(a, s, st);
    case MODE_NN: return launch_g<MODE_NN>(a, s, st);
    default: return cudaErrorInvalidValue;
    }
}

int force_fp64_ctas_per_sm(int groups, int mode)
{
    switch (mode) {
    case MODE_ACC_JERK_POT: return occ_g<MODE_ACC_JERK_POT>(groups);
    case MODE_ACC_POT: return occ_g<MODE_ACC_POT>(groups);
    case MODE_ADJOINT: return occ_g<MODE_ADJOINT>(groups);
    case MODE_NN: return occ_g<MODE_NN>(groups);
    default: return 0;
    }
}

}  // namespace kirin
