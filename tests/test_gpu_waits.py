"""Bounded waits of the streaming matvec (variants 16..19): a wait that runs out ends the launch
with a status the host reads, and the CUDA context stays usable.

The test holds the producer warps' first copies back (vbk_debug_stream_delay) for longer than
the kernels' 1 s wait limit: the computing warps give up waiting, the launch completes, and the
timed stand-alone operator call reports VBK_ERR_CUDA.  No fault, trap or hang is involved: the
delay itself is bounded and every copy lands before the kernel ends.  A second call without the
delay must then succeed and agree with the oracle's operator."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as w  # noqa: E402
from oracle import vibronic as o  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vbk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2307_13483_gb300 as lib

    return lib


def test_stream_wait_runs_out_and_is_reported(vbk):
    desc = w.ci2d_model(10)
    desc["modes"][1]["n"] = 40  # rows of even length: the streaming variants apply
    model = vbk.Model(desc)
    E = np.array([2.7, 3.1])
    rng = np.random.default_rng(5)
    x = rng.standard_normal((2, 2, model.N)) + 1j * rng.standard_normal((2, 2, model.N))
    xd = torch.tensor(x, device="cuda")
    variant = 16
    vbk.vbk_set_op_timing(model, True)  # the timed call synchronises and reads the wait flag
    vbk.vbk_debug_stream_delay(1500)
    with pytest.raises(vbk.VbkError) as ei:
        vbk.vbk_matvec(model, E, xd, precision=vbk.VBK_FP64, variant=variant)
    assert ei.value.code == 3 and "wait" in str(ei.value), str(ei.value)
    # the context is still usable: the same call without the delay is right
    y = vbk.vbk_matvec(model, E, xd, precision=vbk.VBK_FP64, variant=variant).cpu().numpy()
    vbk.vbk_set_op_timing(model, False)
    for e in range(2):
        A = o.a_matrix(desc, E[e])
        for k in range(2):
            ref = A @ x[e, k]
            assert np.abs(y[e, k] - ref).max() <= 1e-13 * np.abs(ref).max()


def test_stream_delay_out_of_range_is_rejected(vbk):
    with pytest.raises(vbk.VbkError) as ei:
        vbk.vbk_debug_stream_delay(20000)
    assert ei.value.code == 1
