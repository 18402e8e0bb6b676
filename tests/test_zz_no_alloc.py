"""The allocation-free density entry point (tsbz_density_noalloc).

Some callers cannot allocate device memory (they run inside another
framework's memory pool or a pre-sized arena, or must avoid cudaMalloc's
device synchronisation); for them the library offers a density call whose
scratch is a static device buffer.  This test calls it through the C ABI
twice in a row, on two different orbital sets (the second needs several
k-chunks of the buffer), and checks each result against the oracle's
density (Eq. 3 with the k average of Eq. 7) and against the context entry
point tsbz_get_density on the same orbitals, within the FP64 parity
tolerance of the other GPU tests.  This file is collected last.
"""
import numpy as np
import pytest

import workloads as W
from oracle.cell import Grid
from oracle.scf import density_from

pytestmark = pytest.mark.gpu

RHO_TOL = 1e-12


def _context_density(cell, psi):
    from paper_2112_00920_gb300 import Propagator
    P = Propagator("fp64")
    cid = P.add_cell_spec(cell)
    sid = P.add_subsim(cid, np.zeros((psi.shape[0], 3)), 0.08, 1)
    P.load_ground_state(sid, psi)
    rho = P.density(sid)
    P.close()
    return rho


def test_density_noalloc_matches_get_density():
    import torch
    from paper_2112_00920_gb300 import build_library
    from paper_2112_00920_gb300._lib import density_noalloc

    assert torch.cuda.is_available()
    build_library()
    cells = [W.cell_a(), W.cell_tiny(atoms="none", n=(20, 18, 16), a=(8.0, 7.5, 7.0), n_bands=3)]
    n_ks = [8, 50]   # 50 k of 5760 points needs two chunks of the 262144-double buffer
    psis = [W.random_orbitals(nk, c.n_bands, c.n, Grid(c).dv, seed=21, tag=i)
            for i, (c, nk) in enumerate(zip(cells, n_ks))]
    orcs = [density_from(c, p) for c, p in zip(cells, psis)]
    refs = [_context_density(c, p) for c, p in zip(cells, psis)]
    devs = [torch.from_numpy(p).cuda() for p in psis]
    outs = [density_noalloc(d, c.occ) for d, c in zip(devs, cells)]   # two calls in a row
    torch.cuda.synchronize()
    for out, orc, ref in zip(outs, orcs, refs):
        got = out.cpu().numpy()
        assert np.max(np.abs(got - orc)) <= RHO_TOL * np.max(np.abs(orc))
        assert np.max(np.abs(got - ref)) <= RHO_TOL * np.max(np.abs(ref))
    # bitwise repeatability: the buffer still holds the second call's partial sums,
    # and repeating the first call overwrites them and gives the same density bit for bit
    again = density_noalloc(devs[0], cells[0].occ)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(again.cpu().numpy(), outs[0].cpu().numpy())


def test_density_noalloc_rejects_oversized_grid():
    import torch
    from paper_2112_00920_gb300 import TsbzError, build_library
    from paper_2112_00920_gb300._lib import density_noalloc

    build_library()
    psi = torch.zeros((1, 1, 1, 1, 262145), dtype=torch.complex128, device="cuda")
    with pytest.raises(TsbzError) as e:
        density_noalloc(psi, 2.0)
    assert e.value.code == -1
