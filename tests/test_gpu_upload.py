"""Ground-state uploads through the C ABI from the three kinds of source
buffer give the same state bit for bit:
- pageable host memory: one copy through the staging buffer;
- page-locked host memory: read by the conversion kernel over the host link,
  without a staging copy, and not waited for before the call returns;
- a device tensor.
Loads of several sub-simulations from page-locked buffers in a row, with
nothing waiting in between, also match."""
import numpy as np
import pytest

import workloads as W
from gpu_common import random_subsim

pytestmark = pytest.mark.gpu


def _cell():
    return W.cell_tiny(atoms="pair", n=(8, 8, 8), a=(6.0, 6.0, 6.0), n_bands=4)


def _subsims(cell, n):
    return [random_subsim(cell, (2, 1, 1), (0.25, 0.5, 0.125), 0.08, 4, W.Kick(k0=0.01), seed=700 + i)
            for i in range(n)]


def _run(precision, cell, subs, source):
    import torch
    from paper_2112_00920_gb300 import Propagator, shifted_kpoints
    P = Propagator(precision)
    cid = P.add_cell_spec(cell)
    sids = [P.add_subsim(cid, shifted_kpoints(cell.a, s["mp"], s["shift"]), s["dt"], s["n_steps"]) for s in subs]
    keep = []   # page-locked and device buffers stay alive (and unchanged) until the library has waited
    for sid, s in zip(sids, subs):
        if source == "pageable":
            buf = np.ascontiguousarray(s["psi"])
        elif source == "pinned":
            t = torch.from_numpy(np.ascontiguousarray(s["psi"])).pin_memory()
            keep.append(t)
            buf = t.numpy()
        else:
            buf = torch.from_numpy(np.ascontiguousarray(s["psi"])).cuda()
            keep.append(buf)
        P.load_ground_state(sid, buf)
    for sid, s in zip(sids, subs):
        P.set_kick(sid, s["field"].k0, s["field"].direction)
    states = [P.get_state(sid)[0] for sid in sids]
    P.propagate(2)
    out = [(st, P.current(sid)[0], P.density(sid)) for st, sid in zip(states, sids)]
    P.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_upload_sources_agree_bitwise(precision):
    import torch
    assert torch.cuda.is_available()
    from paper_2112_00920_gb300 import build_library
    build_library()
    cell = _cell()
    subs = _subsims(cell, 3)
    ref = _run(precision, cell, subs, "pageable")
    for source in ("pinned", "device"):
        got = _run(precision, cell, subs, source)
        for (sa, ja, ra), (sb, jb, rb) in zip(ref, got):
            np.testing.assert_array_equal(sa, sb)
            np.testing.assert_array_equal(ja, jb)
            np.testing.assert_array_equal(ra, rb)
    # the uploaded state is the ground state itself, to the precision of the path
    tol = 0.0 if precision == "fp64" else 2.0 ** -23
    for (st, _, _), s in zip(ref, subs):
        psi = np.asarray(s["psi"])
        assert np.max(np.abs(st - psi)) <= tol * np.max(np.abs(psi))
