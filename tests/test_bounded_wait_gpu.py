"""The failure path of the tensor-core near field's bounded waits, made to happen without
faulting the GPU: a thread block that holds tensor memory waits on an mbarrier that nothing
arrives on. The wait must give up, the call must report HMAT_ETIMEOUT, and the CUDA context
must stay usable for the next product."""
import time

import pytest

from paper_1805_08998_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1805_08998_gb300 import build_lib
    build_lib.build()
    from paper_1805_08998_gb300 import hmat
    hmat.lib()
    return hmat


def test_bounded_wait_gives_up_and_context_survives(H):
    assert H.hmat_check_bounded_wait(1 << 12) == H.HMAT_ETIMEOUT
    t0 = time.perf_counter()
    assert H.hmat_check_bounded_wait(1 << 18) == H.HMAT_ETIMEOUT  # the near field's own limit
    t_limit = time.perf_counter() - t0
    print(f"a wait at the near field's limit (2^18 polls) gives up after {t_limit:.3f} s")
    assert t_limit < 5.0
    for bad in (0, -1, (1 << 22) + 1):
        assert H.hmat_check_bounded_wait(bad) == H.HMAT_EINVAL
    # the context is still usable: an FP32 product, whose near field runs on the tensor cores
    P = inputs.points(inputs.PTS_CUBE, 2, 600, 0)
    A = H.hmat_build(P, H.K_EXP, leaf_size=32, eta=1.0, aca_eps=1e-8, factor_prec=32)
    C = H.hmat_multiply(A, A, 1e-6, mode=H.MODE_MIXED, seed=1)
    assert C.last_status == H.HMAT_OK and C.stats()["n_near"] > 0
