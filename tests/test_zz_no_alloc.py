"""The allocation-free operator entry point against the allocating one (GPU).

ibfem_apply_operator_noalloc serves callers that cannot allocate device memory (their own
pool owns the GPU, or cudaMalloc's device synchronisation is off-limits); it keeps its only
scratch in a static device array.  This file is collected last so that a failure here
never hides the other tests' results.
"""
import numpy as np
import pytest

from helpers import SMALL_CASES, gpu_solver, rel_l2
from paper_2501_19013_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-13   # same bound as the operator parity test


def _inputs(s, w):
    from paper_2501_19013_gb300 import ibfem as ib
    dim, p = w.dim, w.p
    nc = s.ncomp
    n = [int(v) for v in w.n[:dim]]
    n_elem = int(np.prod(n))
    cut = s.cut_cells()
    cls = np.full(n_elem, 2, dtype=np.uint8)
    cls[cut] = 1
    for e in range(n_elem):
        if cls[e] == 1:
            continue
        try:
            s.element(e)
        except ib.IbfemError as err:
            assert err.code == ib.ERR_ARG
            cls[e] = 0
    cut_index = np.full(n_elem, -1, dtype=np.int32)
    cut_index[cut] = np.arange(len(cut), dtype=np.int32)
    K_ref = s.element(int(np.nonzero(cls == 2)[0][0]))[0]
    K_cut = np.stack([s.element(int(e))[0] for e in cut]) if len(cut) else np.zeros((1, 1, 1))
    lat = [k * p + 1 for k in n]
    used = np.zeros(int(np.prod(lat)), dtype=bool)
    for e in np.nonzero(cls != 0)[0]:
        ex, ey = e % n[0], (e // n[0]) % n[1]
        ez = e // (n[0] * n[1]) if dim == 3 else 0
        for c in range(p + 1 if dim == 3 else 1):
            for b in range(p + 1):
                for a in range(p + 1):
                    g = ex * p + a + lat[0] * ((ey * p + b) + lat[1] * (ez * p + c if dim == 3 else 0))
                    used[g] = True
    kept_nodes = np.nonzero(used)[0]
    kept_dofs = (kept_nodes[:, None] * nc + np.arange(nc)[None, :]).ravel()
    return dict(dim=dim, p=p, nc=nc, n=n, cls=cls, cut_index=cut_index, cut=cut, K_ref=K_ref,
                K_cut=K_cut, n_lat_dof=int(np.prod(lat)) * nc, kept_dofs=kept_dofs)


NO_CUT = lambda: W.plate_one_hole().with_(holes=None, name="plate_16x16_p2_no_holes")


@pytest.mark.parametrize("case", ["elastic_evs_ragged", "voxel_3d_evs", "no_cut_cells"])
def test_noalloc_operator_matches_allocating_operator_twice(case):
    """2D plane strain with cut cells, 3D scalar with cut cells, and a grid with no cut cell
    (null cut arrays: the cut-cell kernel is not launched)."""
    import torch
    from paper_2501_19013_gb300 import ibfem as ib

    w = NO_CUT() if case == "no_cut_cells" else SMALL_CASES[case]()
    s = gpu_solver(w)
    d = _inputs(s, w)
    dev = torch.device("cuda", 0)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    cls = t(d["cls"], torch.uint8)
    cut_index = t(d["cut_index"], torch.int32)
    K_ref = t(d["K_ref"], torch.float64)
    if len(d["cut"]):
        cut = t(d["cut"].astype(np.int64), torch.int64)
        K_cut = t(d["K_cut"], torch.float64)
        cut_ptr, kcut_ptr = cut.data_ptr(), K_cut.data_ptr()
    else:
        cut_ptr, kcut_ptr = None, None      # no cut cells: the cut arrays may be null
    rng = np.random.default_rng(11)
    for call in range(2):      # two calls in a row share (and reuse) the static scratch
        x = rng.standard_normal(s.n_dof) * (1.0 + call)
        y_ref = s.apply_operator(x)
        x_lat = np.zeros(d["n_lat_dof"])
        x_lat[d["kept_dofs"]] = x
        xd = t(x_lat, torch.float64)
        yd = torch.full((d["n_lat_dof"],), float("nan"), dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev)
        ib.apply_operator_noalloc(d["dim"], d["p"], d["nc"], d["n"], cls.data_ptr(),
                                  cut_index.data_ptr(), cut_ptr, len(d["cut"]),
                                  K_ref.data_ptr(), kcut_ptr, xd.data_ptr(), yd.data_ptr(),
                                  stream.cuda_stream)
        torch.cuda.synchronize()
        y = yd.cpu().numpy()[d["kept_dofs"]]
        assert rel_l2(y, y_ref) <= TOL
    s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2501_19013_gb300 import ibfem as ib
    with pytest.raises(ib.IbfemError) as err:
        # 2^19 cut cells of 9 DOFs exceed the static scratch; rejected before any launch
        ib.apply_operator_noalloc(2, 2, 1, [1024, 1024], 1, 1, 1, 1 << 19, 1, 1, 1, 1, None)
    assert err.value.code == ib.ERR_ARG
    assert "the static scratch" in str(err.value)
