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
