"""The fifth-generation tensor-core building blocks (tcgen05: tensor-memory
allocation, A operand in tensor memory, B in shared memory through a matrix
descriptor, single-thread MMA issue, mbarrier completion) against a host
product: D = A B^T (128 x 32, K = 16) with the three-product TF32 split that
the projector contractions use, about 2^-21 relative per product."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_umma_three_product_tf32_gemm():
    import torch
    assert torch.cuda.is_available()
    from paper_2112_00920_gb300 import build_library
    from paper_2112_00920_gb300._lib import selftest_umma
    build_library()
    rng = np.random.default_rng(2112)
    a = rng.standard_normal((128, 16)).astype(np.float32)
    b = rng.standard_normal((32, 16)).astype(np.float32)
    ref = a.astype(np.float64) @ b.astype(np.float64).T
    scale = np.max(np.abs(ref))
    errs = {}
    for swap in (False, True):
        rc, st, d = selftest_umma(0, a, b, swap_lbo_sbo=swap)
        assert rc == 0 and st == 0, (rc, st)
        errs[swap] = float(np.max(np.abs(d - ref)) / scale)
    print("tcgen05 three-product TF32 GEMM, max error / max |D|: descriptor as used", errs[False],
          "offsets exchanged", errs[True])
    assert errs[False] <= 2e-6
    # the same call again: the tensor memory of the first call was released
    rc, st, d2 = selftest_umma(0, a, b)
    assert rc == 0 and np.array_equal(d2, selftest_umma(0, a, b)[2])
