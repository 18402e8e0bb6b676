"""GPU: uneven batches in one context, and the autotuner.

Sub-simulations of different cells (the 16^3 cell A on the fused stage
kernels, the 32^3, 64-atom cell B on the slab z-march stage in single
precision and the point-parallel kernels in FP64), different
subgrid sizes and different step budgets advance together through the C ABI;
each is compared with the oracle run on its own.  The autotuner's trial steps
must leave the state bit for bit as it was, and every kernel variant it can
choose must meet the same parity bars as the default.
"""
import numpy as np
import pytest

import workloads as W
from oracle.cell import Grid

from gpu_common import FP32_J_TOL, FP32_RHO_TOL, FP64_J_TOL, FP64_RHO_TOL, compare, oracle_run, random_subsim

pytestmark = pytest.mark.gpu
BARS = {"fp64": (FP64_J_TOL, FP64_RHO_TOL), "fp32": (FP32_J_TOL, FP32_RHO_TOL), "fp32_tc": (FP32_J_TOL, FP32_RHO_TOL)}


@pytest.fixture(scope="module", autouse=True)
def built_library():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2112_00920_gb300 import build_library
    build_library()


def _context(precision, groups, graphs=False):
    """groups: list of (cell, [subsim dicts]); returns (propagator, ids per subsim in order)."""
    from paper_2112_00920_gb300 import Propagator, shifted_kpoints
    P = Propagator(precision)
    P.set_graphs(graphs)
    ids = []
    for cell, subs in groups:
        cid = P.add_cell_spec(cell)
        for s in subs:
            ids.append((cid, P.add_subsim(cid, shifted_kpoints(cell.a, s["mp"], s["shift"]), s["dt"],
                                          s["n_steps"]), cell, s))
    for _, sid, _, s in ids:
        P.load_ground_state(sid, s["psi"])
        P.set_kick(sid, s["field"].k0, s["field"].direction)
    return P, ids


def _gpu_result(P, sid):
    J, j0 = P.current(sid)
    return dict(J=J, J0m=j0, rho=P.density(sid), norms=P.norms(sid))


_ORACLE = {}


def _oracle(key, cell, s):
    if key not in _ORACLE:
        _ORACLE[key] = oracle_run(cell, s)
    return _ORACLE[key]


def _tiny():
    return W.cell_tiny(atoms="pair", n=(8, 8, 8), a=(6.0, 6.0, 6.0), n_bands=4)


@pytest.mark.parametrize("precision,graphs", [("fp64", False), ("fp32", False), ("fp32", True)])
def test_step_budgets(precision, graphs):
    """Budgets 3 and 6 in one context: propagate(4) twice leaves the first at 3
    steps and the second at 6, each equal to the oracle run of its own length."""
    cell = _tiny()
    s0 = random_subsim(cell, (2, 1, 1), (0.25, 0.5, 0.0), 0.08, 3, W.Kick(k0=0.01), seed=31)
    s1 = random_subsim(cell, (1, 2, 2), (0.5, 0.25, 0.75), 0.08, 6, W.Kick(k0=0.02), seed=32)
    P, ids = _context(precision, [(cell, [s0, s1])], graphs=graphs)
    P.propagate(4)
    assert [P.step(i[1]) for i in ids] == [3, 4]
    P.propagate(4)
    assert [P.step(i[1]) for i in ids] == [3, 6]
    jt, rt = BARS[precision]
    for key, (_, sid, c, s) in zip(("b0", "b1"), ids):
        errs = compare(_gpu_result(P, sid), _oracle(key, c, s), jt, rt)
        print(precision, graphs, key, errs)
    P.close()


def _mixed_groups(nb_b=8):
    ca, cb = W.cell_a(), W.cell_b(n_bands=nb_b)
    a_subs = [random_subsim(ca, (2, 1, 1), (0.125, 0.375, 0.625), 0.08, 4, W.Kick(k0=0.005), seed=41),
              random_subsim(ca, (1, 1, 3), (0.7, 0.2, 0.9), 0.08, 2, W.Kick(k0=0.0003), seed=42)]
    b_subs = [random_subsim(cb, (2, 1, 1), (0.3, 0.6, 0.1), 0.08, 3, W.Kick(k0=0.002), seed=43),
              random_subsim(cb, (1, 1, 2), (0.8, 0.4, 0.55), 0.08, 4, W.Kick(k0=0.0001), seed=45)]
    return [(ca, a_subs), (cb, b_subs)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mixed_cells_uneven(precision):
    """Two sub-simulations of cell A (16^3, 16 bands) and two of cell B (32^3, 64
    atoms; 8 of its bands) with subgrids of 2, 3, 2 and 2 k-points, kicks 5e-3 /
    3e-4 / 2e-3 / 1e-4 and budgets 4, 2, 3, 4 in one context; every sub-simulation
    matches its own oracle run."""
    groups = _mixed_groups()
    P, ids = _context(precision, groups)
    P.propagate(4)
    assert [P.step(i[1]) for i in ids] == [4, 2, 3, 4]
    jt, rt = BARS[precision]
    for n, (_, sid, c, s) in enumerate(ids):
        errs = compare(_gpu_result(P, sid), _oracle(("mixed", n), c, s), jt, rt)
        print(precision, "sub", n, c.name, errs)
    P.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cell_b_full_bands(precision):
    """The 2x2x2 supercell at its full size: 32^3 grid, 64 atoms (256 projectors),
    128 bands, one k-point, two steps."""
    cb = W.cell_b()
    s = random_subsim(cb, (1, 1, 1), (0.3, 0.1, 0.7), 0.08, 2, W.Kick(k0=0.005), seed=44)
    P, ids = _context(precision, [(cb, [s])])
    P.propagate(2)
    jt, rt = BARS[precision]
    errs = compare(_gpu_result(P, ids[0][1]), _oracle("cellB128", cb, s), jt, rt)
    print(precision, "cell B 128 bands", errs)
    P.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_autotune_restores_state_and_keeps_parity(precision):
    """After one step, autotune the mixed context: orbitals, step counts,
    densities and norms are bit for bit unchanged; then two more steps with
    the chosen variants still match the oracle."""
    groups = _mixed_groups()
    # every budget at 3 steps so that all sub-simulations are compared at 3
    for _, subs in groups:
        for s in subs:
            s["n_steps"] = 3
    P, ids = _context(precision, groups)
    P.propagate(1)
    before = [(P.get_state(sid), P.density(sid), P.norms(sid), P.current(sid)) for _, sid, _, _ in ids]
    n = P.autotune(budget_ms=60000)
    assert n >= 6   # cell A: 3 or more variants; cell B: 3 (FP64) or 4 (FP32)
    for (_, sid, _, _), (st, rho, nr, cur) in zip(ids, before):
        st2 = P.get_state(sid)
        assert st2[1] == st[1] == 1
        assert np.array_equal(st2[0], st[0])
        assert np.array_equal(P.density(sid), rho)
        assert np.array_equal(P.norms(sid), nr)
        assert np.array_equal(P.current(sid)[0], cur[0])
    for cid in sorted({i[0] for i in ids}):
        v, nv, ms = P.variant(cid)
        assert 0 <= v < nv and nv >= 2 and all(t > 0 for t in ms)
        print(precision, "cell", cid, "variant", v, "of", nv, "ms/step", ms)
    P.propagate(2)
    jt, rt = BARS[precision]
    for n_, (_, sid, c, s) in enumerate(ids):
        errs = compare(_gpu_result(P, sid), oracle_run(c, s), jt, rt)
        print(precision, "after autotune, sub", n_, errs)
    P.close()


def _cube16(frac):
    return W.cell_tiny(atoms="pair", n=(16, 16, 16), a=(8.0, 8.5, 9.0), n_bands=4,
                       atom_frac=np.asarray(frac, dtype=np.float64))


# 16^3 cells whose atoms form z groups of one atom (whole step runs), no usable
# groups (6 distinct z planes) or a group of three (both take the per-atom kernels)
_Z_ONE = [[0.1, 0.2, 0.3], [0.55, 0.6, 0.7]]
_Z_SIX = [[0.05 * i + 0.1, 0.13 * i, 0.11 * i + 0.02] for i in range(6)]
_Z_THREE = [[0.0, 0.0, 0.25], [0.5, 0.25, 0.25], [0.25, 0.75, 0.25]]

VARIANT_CASES = [
    # (precision, cell factory, mp, number of variants)
    # whole step (tcgen05) / fused stage (tcgen05) / CUDA-core z-march / whole step (mma.sync)
    ("fp32", W.cell_a, (2, 1, 1), 4),
    ("fp32", lambda: _cube16(_Z_ONE), (2, 1, 1), 4),  # z groups of one atom
    ("fp32", lambda: _cube16(_Z_SIX), (2, 1, 1), 2),  # per-atom fused stage / z-march
    ("fp32", lambda: _cube16(_Z_THREE), (1, 2, 1), 2),
    ("fp32", _tiny, (2, 2, 1), 2),                    # bulk-staged 8^3 stage / z-march
    ("fp32", lambda: W.cell_tiny(atoms="offgrid", n=(10, 12, 14), a=(7.0, 8.0, 9.0), n_bands=3), (3, 1, 1), 3),
    # 32-point rows: slab z-march stage / point-parallel with 4, 16, 8 bands per chunk
    ("fp32", lambda: W.cell_b(n_bands=4), (1, 1, 2), 4),   # 64 atoms in 8 z groups
    # (grid spacings near cell B's 0.64 bohr: dt = 0.08 stays inside the Taylor-4 stability bound)
    ("fp32", lambda: W.cell_tiny(atoms="offgrid", n=(32, 16, 24), a=(20.0, 10.0, 15.0), n_bands=3), (2, 1, 1), 4),
    ("fp32", lambda: W.cell_tiny(atoms="none", n=(32, 16, 16), a=(20.0, 10.0, 10.5), n_bands=3), (1, 2, 1), 4),
    ("fp64", _tiny, (2, 2, 1), 3),                    # point-parallel: 8, 4, 16 bands per chunk
    ("fp32_tc", W.cell_a, (2, 1, 1), 3),              # bulk-staged stencil stage (t; t, V, psi) / halo-plane z-march
    ("fp32_tc", lambda: W.cell_tiny(atoms="offgrid", n=(10, 12, 16), a=(7.0, 8.0, 9.0), n_bands=3), (3, 1, 1), 1),
]


@pytest.mark.parametrize("case", range(len(VARIANT_CASES)))
def test_every_variant_parity(case):
    precision, make, mp, nv = VARIANT_CASES[case]
    cell = make()
    s = random_subsim(cell, mp, (0.25, 0.5, 0.125), 0.08, 4, W.Kick(k0=0.01), seed=50 + case)
    o = oracle_run(cell, s)
    jt, rt = BARS[precision]
    for v in range(nv):
        P, ids = _context(precision, [(cell, [s])])
        cid = ids[0][0]
        assert P.variant(cid)[1] == nv
        P.set_variant(cid, v)
        P.propagate(4)
        errs = compare(_gpu_result(P, ids[0][1]), o, jt, rt)
        print(precision, cell.name, "variant", v, errs)
        P.close()
    with pytest.raises(Exception):
        P, ids = _context(precision, [(cell, [s])])
        try:
            P.set_variant(ids[0][0], nv)
        finally:
            P.close()


def test_mixed_graph_replay_bitwise():
    """The mixed cell-A / cell-B batch in single precision (whole-step kernel on
    cell A, slab stage and cluster projections on cell B) gives the same orbitals
    and currents bit for bit whether its steps are launched directly or replayed
    from the captured graph, and twice in a row: every reduction runs in a fixed
    order."""
    out = []
    for graphs in (False, True, True):
        P, ids = _context("fp32", _mixed_groups(), graphs=graphs)
        P.propagate(2)
        P.propagate(2)
        out.append([(P.current(sid)[0], P.get_state(sid)[0], P.density(sid)) for _, sid, _, _ in ids])
        P.close()
    for run in out[1:]:
        for (ja, sa, ra), (jb, sb, rb) in zip(out[0], run):
            np.testing.assert_array_equal(ja, jb)
            np.testing.assert_array_equal(sa, sb)
            np.testing.assert_array_equal(ra, rb)
