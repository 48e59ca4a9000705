"""The launch-shape autotuner: it installs a table the library then follows, and results stay exact."""
import numpy as np
import pytest

import oracle
from paper_0707_0438_gb300 import abi, autotune, workloads
from tests.gpu_util import assert_parity

pytestmark = pytest.mark.gpu


def test_autotuned_table_is_used_and_correct(kirin_lib, tmp_path):
    import torch
    p = workloads.plummer(8192, 1002, eps=1e-3)
    with abi.Kirin(p.n, p.eps, stream=torch.cuda.current_stream().cuda_stream) as k:
        k.set_j_particles(p.m, p.x, p.v)
        entries = autotune.tune(k, p.n, reps=2, cache=str(tmp_path / "t.json"), device_name="test")
        assert entries and entries[-1][0] == p.n
        assert all(a[0] < b[0] for a, b in zip(entries, entries[1:]))
        for n_i_max, g, s, _ in entries:
            if n_i_max <= 8:  # blocks this small go to the tiny-block kernel whatever the table says
                assert k.get_launch(n_i_max)[0] == 0
            else:
                assert k.get_launch(n_i_max) == (g, min(s, (p.n + 127) // 128))
        for n_i in (1, 37, 1000, 8192):
            il = workloads.i_subset(p.n, n_i, n_i)
            got = k.forces(il)
            assert_parity(got, oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=il), "mixed", f"tuned n_i={n_i}")
        # the cache is reused
        again = autotune.tune(k, p.n, cache=str(tmp_path / "t.json"), device_name="test")
        assert [tuple(e[:3]) for e in again] == [tuple(e[:3]) for e in entries]
        k.set_launch_table([])
        assert k.get_launch(8192) != (0, 0)


def test_launch_table_rejects_bad_entries(kirin_lib):
    p = workloads.plummer(100, 1, eps=0.01)
    with abi.Kirin(p.n, p.eps) as k:
        for bad in ([(10, 3, 1)], [(10, 1, 0)], [(10, 1, 1), (5, 1, 1)], [(10, 1, 2000)]):
            with pytest.raises(abi.KirinError) as e:
                k.set_launch_table(bad)
            assert e.value.code == abi.KIRIN_EINVAL


def test_tables_per_call_kind(kirin_lib, tmp_path):
    """Acceleration-and-potential and adjoint calls follow their own tables (tuned here for a small
    sphere), the full force calls keep theirs, and the results do not change."""
    import torch
    dev = torch.device("cuda:0")
    p = workloads.plummer(3000, 17, masses="lognormal", eps=0.01)
    m = torch.tensor(p.m, device=dev)
    x = torch.tensor(p.x, device=dev)
    with abi.Kirin(p.n, p.eps, stream=torch.cuda.current_stream().cuda_stream) as k:
        k.set_j_particles(p.m, p.x, p.v)
        forces = k.get_launch(p.n)
        acc = torch.empty_like(x)
        pot = torch.empty_like(m)
        k.accel_dev(m, x, acc, pot)
        k.sync()
        before = acc.cpu().numpy()
        e = autotune.tune_full(k, m, x, "acc_pot", reps=1, cache=str(tmp_path / "t.json"), device_name="test")
        assert len(e) == 1 and e[0][0] == p.n
        assert k.get_launch(p.n, abi.KIRIN_CALL_ACC_POT) == (e[0][1], min(e[0][2], (p.n + 127) // 128))
        assert k.get_launch(p.n) == forces
        k.set_launch_table([(p.n, 8, 3)], abi.KIRIN_CALL_ADJOINT)
        assert k.get_launch(p.n, abi.KIRIN_CALL_ADJOINT) == (8, 3)
        k.accel_dev(m, x, acc, pot)
        k.sync()
        ra, rp = oracle.acc_pot(p.m, p.x, p.eps)
        assert np.median(np.linalg.norm(acc.cpu().numpy() - ra, axis=1) / np.linalg.norm(ra, axis=1)) <= 1e-6
        assert np.max(np.abs(acc.cpu().numpy() - before)) <= 1e-6 * np.max(np.abs(before))
        with pytest.raises(abi.KirinError):
            k.set_launch_table([(p.n, 4, 2)], 3)
        # a stored table for each kind is installed together with the others
        assert autotune.install(k, p.n, "test", "mixed", path=str(tmp_path / "t.json")) is False
        assert k.get_launch(p.n, abi.KIRIN_CALL_ACC_POT) == (e[0][1], min(e[0][2], (p.n + 127) // 128))
