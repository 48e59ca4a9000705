"""The integer-built FP64 -> FP32 conversions of the mixed j images (csrc/f32_pack.cuh) against
IEEE round-to-nearest-even conversions (numpy's, on the host).

The images hold each coordinate as hi = RN32(x), lo = RN32(x - hi) (Sect. 3.1: the j-particle
data the force kernels read, here in double-single), and mass and velocity as RN32. The step
kernels build these words from the operands' bits instead of the FP64 conversion instruction;
the words must be the same bits. The header compiles as plain C++, so g++ builds it here.

Cases that would catch a plausible slip: ties with an even and an odd kept word (round half to
even), a fraction of all ones that carries into the exponent, the first and last exponent of
each range, zero of both signs, tiny, huge and non-finite values (the conversion path), and a
few hundred thousand random doubles over the whole exponent range."""
import pathlib
import shutil
import subprocess

import numpy as np
import pytest

CSRC = pathlib.Path(__file__).resolve().parents[1] / "paper_0707_0438_gb300" / "csrc"

DRIVER = r"""
#include <stdio.h>
#include <stdlib.h>
#include "f32_pack.cuh"
int main(int argc, char **argv)
{
    FILE *fi = fopen(argv[1], "rb"), *fo = fopen(argv[2], "wb");
    double v;
    while (fread(&v, sizeof v, 1, fi) == 1) {
        float hi, lo;
        kirin::f32pack::split(v, hi, lo);
        const float c = kirin::f32pack::to_f32(v);
        const unsigned char fin = kirin::f32pack::finite(v);
        fwrite(&hi, 4, 1, fo);
        fwrite(&lo, 4, 1, fo);
        fwrite(&c, 4, 1, fo);
        fwrite(&fin, 1, 1, fo);
    }
    fclose(fi);
    fclose(fo);
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("f32pack")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    exe = d / "drv"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", str(CSRC), str(src), "-o",
                    str(exe)], check=True)
    return exe, d


def _run(driver, values):
    exe, d = driver
    values = np.ascontiguousarray(values, dtype=np.float64)
    (d / "in.bin").write_bytes(values.tobytes())
    subprocess.run([str(exe), str(d / "in.bin"), str(d / "out.bin")], check=True)
    rec = np.frombuffer((d / "out.bin").read_bytes(),
                        dtype=np.dtype([("hi", "<u4"), ("lo", "<u4"), ("c", "<u4"), ("fin", "u1")]))
    assert rec.shape == values.shape
    return rec


def _expected(values):
    with np.errstate(over="ignore", invalid="ignore"):
        hi = values.astype(np.float32)
        lo = (values - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def _from_bits(bits):
    return np.asarray(bits, dtype=np.uint64).view(np.float64)


def _edge_values():
    v = []
    # ties and near-ties in the 29 dropped bits, kept word even and odd, both signs
    for e in (949, 1000, 1023, 1030, 1149, 897, 1150):
        for keep in (0, 1, 2, 3, (1 << 23) - 2, (1 << 23) - 1):
            for rem in (0, 1, 0x0FFFFFFF, 0x10000000, 0x10000001, 0x1FFFFFFF):
                for s in (0, 1):
                    v.append((s << 63) | (e << 52) | (keep << 29) | rem)
    # the first and last exponents of the two ranges and their neighbours
    for e in (0, 1, 895, 896, 897, 898, 947, 948, 949, 950, 1148, 1149, 1150, 1151, 2046):
        for frac in (0, 1, (1 << 52) - 1, 0x8000000000000, 0x10000000):
            v.append((e << 52) | frac)
            v.append((1 << 63) | (e << 52) | frac)
    bits = np.array(v, dtype=np.uint64)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, 2.2250738585072014e-308,
                        1.0, -1.0, 0.5, 1e4, -1e4, 1.0 / 3.0, np.pi, 3.4028234663852886e38,
                        3.4028235677973366e38, 3.402823669209385e38, 1.1754943508222875e-38,
                        1.1754942106924411e-38, 2.0 ** -74, 2.0 ** -75, 2.0 ** 127, 2.0 ** 128])
    return np.concatenate([_from_bits(bits), special])


def _random_values(seed, count):
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 1 << 63, size=count, dtype=np.uint64) | (
        rng.integers(0, 2, size=count, dtype=np.uint64) << np.uint64(63))
    # half of them with exponents near the image's working range (positions, velocities, masses)
    e = rng.integers(900, 1100, size=count // 2, dtype=np.uint64)
    bits[: count // 2] = (bits[: count // 2] & ~np.uint64(0x7FF << 52)) | (e << np.uint64(52))
    return np.concatenate([_from_bits(bits), rng.standard_normal(count // 4),
                           rng.lognormal(0.0, 3.0, count // 4) * 1e-6])


@pytest.mark.parametrize("which", ["edges", "random"])
def test_split_and_rn32_match_the_conversions_bit_for_bit(driver, which):
    values = _edge_values() if which == "edges" else _random_values(20241204, 200000)
    rec = _run(driver, values)
    hi, lo = _expected(values)
    nan = np.isnan(values)
    ok = ~nan
    np.testing.assert_array_equal(rec["hi"][ok], hi.view(np.uint32)[ok])
    np.testing.assert_array_equal(rec["lo"][ok], lo.view(np.uint32)[ok])
    np.testing.assert_array_equal(rec["c"][ok], hi.view(np.uint32)[ok])
    # NaN converts to a NaN
    assert np.isnan(rec["hi"][nan].view(np.float32)).all() and np.isnan(rec["c"][nan].view(np.float32)).all()
    np.testing.assert_array_equal(rec["fin"].astype(bool), np.isfinite(values))


def test_split_reconstructs_the_double_to_48_bits(driver):
    """hi + lo carries the coordinate to within 2^-48 of itself (the double-single image's
    precision), which a wrong sign or scale of the low word would break."""
    rng = np.random.default_rng(7)
    values = rng.uniform(-2.0, 2.0, 50000) * 10.0 ** rng.integers(-6, 4, 50000)
    rec = _run(driver, values)
    back = rec["hi"].view(np.float32).astype(np.float64) + rec["lo"].view(np.float32).astype(np.float64)
    assert np.all(np.abs(back - values) <= np.abs(values) * 2.0 ** -48)
