"""The slab split with the library's own local solves (FP64 on the CUDA
path): P slabs of one grid solved one after another on this GPU, with the
same ghost rows, exchanges and termination as the distributed form (whose
protocol tests/test_slab_cpu.py runs over gloo ranks).  The slabs put
together must be the oracle's whole-grid solution within the FP64
tolerance, with +inf at the same nodes."""
import numpy as np
import pytest

from paper_1110_6220_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


@pytest.fixture(scope="module")
def slab():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_6220_gb300 import build
    build.build()
    from paper_1110_6220_gb300 import slab as s
    return s


@pytest.mark.parametrize("P", [2, 4])
def test_slabs_with_library_solves_match_the_whole_grid(slab, orc, P):
    for I in [W.sin_point(257), W.checker_maze(257, seed=3, n_walls=6, n_src=3)]:
        V = orc.fmm(I.F, I.h, I.si, I.sj, I.sq)
        U, rounds = slab.solve_slabs(I.F, I.h, I.si, I.sj, I.sq, P, cell_k=8)
        fin = np.isfinite(V)
        assert (np.isfinite(U) == fin).all(), I.name
        err = np.abs(U[fin] - V[fin]).max() / np.abs(V[fin]).max()
        assert err <= TOL64, (I.name, P, err)
        assert rounds >= 2
