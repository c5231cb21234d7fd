"""Multi-rank (replica) aggregation of bench.py on CPU with the gloo backend, world size 2."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    step_ms = [2.0, 3.0][rank]          # rank 1 is the slower replica
    n_dof = [1000, 1000][rank]
    out[rank] = bench.aggregate_replicas(step_ms, n_dof, world)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_takes_slowest_rank_and_all_dofs():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        step_ms, value = out[r]
        assert step_ms == pytest.approx(3.0)
        assert value == pytest.approx(2000 / 3e-3)


def test_single_rank_aggregation():
    import bench
    step_ms, value = bench.aggregate_replicas(2.0, 1000, 1)
    assert step_ms == 2.0 and value == pytest.approx(1000 / 2e-3)


def test_accuracy_against_fp64_on_fake_runs():
    """The bench's accuracy table: final-field rel-L2 and the observer error e_100 / e_N
    of each variant against the FP64 path of the same scheme and stabilisation; none where
    that scheme has no FP64 run."""
    import numpy as np
    import bench

    class Info:
        ncomp = 2

        def __init__(self, precision):
            self.precision = precision

    t = np.linspace(0.0, 1.0, 1001)
    ref = np.stack([np.sin(5 * t + i) for i in range(6)], axis=1)
    u = np.linspace(1.0, 2.0, 50)
    results = {
        "fp64": dict(scheme="cdm", stab="evs", u_end=u, series=ref, info=Info(0)),
        "exact": dict(scheme="cdm", stab="evs", u_end=u * (1 + 3e-6), series=ref * (1 + 2e-6), info=Info(1)),
        "imex:exact": dict(scheme="imex", stab="none", u_end=u * (1 - 5e-6), series=ref, info=Info(1)),
        "cons:exact": dict(scheme="cdm_consistent", stab="evs", u_end=u, series=ref, info=Info(1)),
    }
    bench.accuracy_against_fp64(results)
    assert results["fp64"]["rel_l2"] == 0.0 and results["fp64"]["e_obs"]["e_100"] == 0.0
    assert abs(results["exact"]["rel_l2"] - 3e-6) < 1e-12
    assert abs(results["exact"]["e_obs"]["e_100"] - 2e-6) < 1e-12
    assert abs(results["exact"]["e_obs"]["e_1000"] - 2e-6) < 1e-12
    assert results["exact"]["e_obs"]["e_N"] == results["exact"]["e_obs"]["e_1000"]
    assert results["exact"]["e_obs"]["observers_left_out"] == 0
    assert len(results["exact"]["e_obs"]["e_1000_per_observer"]) == 3
    # no FP64 run of IMEX or of the consistent mass: nothing to compare with
    assert results["imex:exact"]["rel_l2"] is None and results["imex:exact"]["e_obs"] is None
    assert results["cons:exact"]["rel_l2"] is None
    results["imex"] = dict(scheme="imex", stab="none", u_end=u, series=ref, info=Info(0))
    bench.accuracy_against_fp64(results)
    assert abs(results["imex:exact"]["rel_l2"] - 5e-6) < 1e-12
    assert results["imex:exact"]["e_obs"]["e_N"] == 0.0
    del results["fp64"]
    bench.accuracy_against_fp64(results)
    assert results["exact"]["rel_l2"] is None


def test_qualification_needs_both_accuracy_measures():
    """A variant counts toward time-to-accuracy only if its final-field rel-L2 and its
    observer error e_N are both within 1e-4 of the FP64 path."""
    import bench
    ok = {"rel_l2": 2e-6, "e_obs": {"e_N": 3e-6}}
    bad_obs = {"rel_l2": 2e-6, "e_obs": {"e_N": 0.5}}
    bad_field = {"rel_l2": 2e-3, "e_obs": {"e_N": 1e-6}}
    assert bench.qualifies(ok) and not bench.qualifies(bad_obs) and not bench.qualifies(bad_field)
    assert not bench.qualifies({"rel_l2": None, "e_obs": None})
    assert bench.qualifies({"rel_l2": 0.0, "e_obs": None})


def test_algorithmic_bytes_follow_the_roofline_model():
    """32 B per DOF + packed symmetric FP64 cut matrices + 4 B per cell; the plate benchmark
    (1 873 378 DOFs, 1 281 distinct cut matrices of n_loc = 50, 256^2 cells) moves 73.3 MB."""
    import bench

    class Inf:
        n_dof, n_loc, n_cut_matrices = 1873378, 50, 1281

    class Wl:
        dim, n = 2, (256, 256)

    b = bench.algorithmic_bytes(Inf(), Wl())
    assert b == 32 * 1873378 + 1281 * 50 * 51 * 4 + 4 * 65536
    assert abs(b - 73.3e6) < 0.05e6


def test_imex_solve_roofline_counts_the_factor():
    """The c-set solve is measured on the survey's model: both sweeps read L once (8 B value
    and 4 B index per entry) plus 48 B per c-DOF of vectors."""
    import bench

    class Inf:
        n_dof, n_loc, n_cut_matrices, nnz_L, n_c = 2092915, 16, 2564, 592535, 30765

    class Wl:
        dim, n, name = 2, (512, 512), "plate_holes_imex_512x512_p3"

    r = bench.roofline("fp64", "imex_solve", 0.128, Inf(), Wl(), {"hbm_gbs": 6800.0}, {})
    byts = 2 * 592535 * 12 + 48 * 30765
    assert r["bound"] == "hbm" and r["kernel"] == "imex_solve"
    assert abs(r["achieved"] - byts / 0.128e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 6800.0) < 1e-15
