"""Failure detection without a GPU fault: a bounded device wait that runs out.

The single-stream encoder places each chunk group's bytes by a decoupled
look-back over the groups before it, a wait bounded by a poll limit.  Here
the context's failure test makes the encoder start its ticket at 1, so chunk
group 0 is never encoded and never publishes its offset: every group that
looks back to it waits a few hundred polls, gives up, and records
SPRINTZ_ERR_TIMEOUT.  The kernel returns (the call completes), the error
reaches the host through sprintz_get_status, and the context stays usable:
the next compression, with the test switched off, writes the oracle's
bytes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def spz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_02515_gb300 import _build
    _build.build()
    import paper_1808_02515_gb300.sprintz as spz
    return spz


@pytest.mark.parametrize("D,fc", [(8, 1), (3, 0), (40, 1)])
def test_lookback_wait_runs_out_and_is_reported(spz, oracle_mod, D, fc):
    import time
    from paper_1808_02515_gb300 import synth
    x = synth.sensor_u16(64 * 1024 + 5, D, seed=70 + D)
    xt = torch.from_numpy(x.view(np.int16)).cuda()
    opts = spz.Opts(forecaster=fc)
    codec = spz.Codec(0)
    try:
        codec.set_failure_test(wait_limit=256, skip_first_group=1)
        t0 = time.perf_counter()
        codec.compress(xt, opts)
        torch.cuda.synchronize()  # the kernel returned
        waited = time.perf_counter() - t0
        assert codec.status() == spz.ERR_TIMEOUT
        assert waited < 30.0
        codec.set_failure_test(0, 0)
        dst, size = codec.compress(xt, opts)
        torch.cuda.synchronize()
        assert codec.status() == spz.OK
        n = int(size.item())
        ref = oracle_mod.compress(x, forecaster=fc, huffman=0, group_blocks=2, learn_shift=1, chunk_rows=1024,
                                  huff_chunks=64)
        assert np.array_equal(dst[:n].cpu().numpy(), ref)
    finally:
        codec.close()


def test_failure_test_arguments_checked(spz):
    codec = spz.Codec(0)
    try:
        with pytest.raises(spz.SprintzError):
            codec.set_failure_test(0, 2)
    finally:
        codec.close()
