"""Failure detection without a GPU fault: every wait inside the tensor-core
Gram kernel is bounded.  The test makes one wait run out on purpose (the
launch waits on a barrier phase that nothing completes, with a 200 us bound),
then checks that the call returned, that mdn_train_status reports the
expired wait once, and that the next launch with the default bound gives the
same Gram sums as a launch before the failure (the context stays usable and
the kernel freed its tensor memory)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mdn():
    import paper_1802_06130_gb300 as m
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    m.build()
    m.lib()
    return m


@pytest.mark.parametrize("prec", ["tf32", "bf16", "split"])
def test_expired_wait_is_reported_and_the_next_launch_is_correct(mdn, prec):
    p = {"tf32": mdn.GRAM_TF32, "bf16": mdn.GRAM_BF16, "split": mdn.GRAM_SPLIT_BF16}[prec]
    pairs = [synth.noisy_pair(192, 160, 700 + i) for i in range(2)]
    Z = torch.tensor(np.stack([a for a, _ in pairs]), device="cuda")
    U = torch.tensor(np.stack([b for _, b in pairs]), device="cuda")
    geom, bp = mdn.Geometry(3, -1, 1), mdn.default_bparams(0)

    def gram():
        g, c, _ = mdn.train_level_filters(Z, None, U, geom, bp, p, solve=False)
        torch.cuda.synchronize()
        return g, c

    assert mdn.train_status() == 0
    g_ref, c_ref = gram()
    assert mdn.train_status() == 0
    try:
        mdn.set_gram_wait_limit(200_000)
        mdn.gram_expire_next_wait(True)
        gram()                                     # returns: the status covers launch checks only
        assert mdn.train_status() == 1             # the device reported the expired wait
        assert mdn.train_status() == 0             # read-and-clear
    finally:
        mdn.set_gram_wait_limit(0)
        mdn.gram_expire_next_wait(False)
    g2, c2 = gram()
    assert mdn.train_status() == 0
    assert torch.equal(c2, c_ref) and int(c2.sum()) == 2 * 192 * 160
    assert torch.equal(g2, g_ref)
