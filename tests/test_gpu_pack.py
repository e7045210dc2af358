"""sprintz_pack: device buffers back to back, their offsets an exclusive scan
taken on the device.  Checked against the host concatenation for buffers of
every size from 0 up and every alignment, for a batch of compressed streams
(their sizes read by the kernel from the batch's size words), and for a
destination that is too small (nothing copied, the error recorded)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def codec():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_02515_gb300 import _build
    _build.build()
    import paper_1808_02515_gb300.sprintz as spz
    c = spz.Codec(0)
    yield c
    c.close()


def test_pack_matches_host_concatenation(codec):
    import paper_1808_02515_gb300.sprintz as spz
    rng = np.random.default_rng(3)
    pool = torch.from_numpy(rng.integers(0, 256, 1 << 25, dtype=np.uint8)).cuda()
    lens = [0, 1, 2, 3, 15, 16, 17, 31, 64, 1000, 4093, 65536 + 7] + [int(v) for v in rng.integers(0, 20000, 1500)]
    starts, pos = [], 0
    for k, n in enumerate(lens):
        pos += k % 19  # every alignment
        starts.append(pos)
        pos += n
    assert pos < pool.numel()
    ptrs = torch.tensor([pool.data_ptr() + s for s in starts], dtype=torch.int64, device="cuda")
    sizes = torch.tensor(lens, dtype=torch.int64, device="cuda")
    total = sum(lens)
    dst = torch.full((total + 5,), 0xEE, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(len(lens) + 1, dtype=torch.int64, device="cuda")
    dst_off = dst[3:]  # an unaligned destination
    codec.pack(ptrs, sizes, dst_off, offs)
    torch.cuda.synchronize()
    assert codec.status() == spz.OK
    host = pool.cpu().numpy()
    want = np.concatenate([host[s:s + n] for s, n in zip(starts, lens)])
    got = dst.cpu().numpy()
    assert np.array_equal(got[3:3 + total], want)
    assert np.all(got[:3] == 0xEE) and np.all(got[3 + total:] == 0xEE)
    assert np.array_equal(offs.cpu().numpy(), np.concatenate([[0], np.cumsum(lens)]))


def test_pack_compressed_batch_and_decode_from_it(codec, oracle_mod):
    import paper_1808_02515_gb300.sprintz as spz
    from paper_1808_02515_gb300 import synth
    xs_h = [synth.batch_stream(i, max_rows=20_000) for i in range(60)]
    xs = [torch.from_numpy(x.view(np.int16) if x.dtype == np.uint16 else x).cuda() for x in xs_h]
    bufs, sizes, _ = codec.compress_batch(xs, spz.Opts())
    torch.cuda.synchronize()
    ptrs = torch.tensor([b.data_ptr() for b in bufs], dtype=torch.int64, device="cuda")
    cap = sum(b.numel() for b in bufs)
    dst = torch.empty(cap, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(len(bufs) + 1, dtype=torch.int64, device="cuda")
    codec.pack(ptrs, sizes, dst, offs)
    torch.cuda.synchronize()
    assert codec.status() == spz.OK
    o = offs.cpu().numpy()
    sz = sizes.cpu().numpy()
    assert np.array_equal(np.diff(o), sz)
    views = [dst[int(o[k]):int(o[k + 1])] for k in range(len(bufs))]
    for x, v in zip(xs_h, views):
        assert np.array_equal(v.cpu().numpy(), oracle_mod.compress(x, forecaster=1))
    infos = [spz.query(v[:64].cpu().numpy().tobytes()) for v in views]
    outs, _ = codec.decompress_batch(views, infos, [int(v) for v in sz])
    torch.cuda.synchronize()
    assert codec.status() == spz.OK
    assert all(torch.equal(a.view(-1), b.view(-1)) for a, b in zip(xs, outs))


def test_pack_too_small_copies_nothing(codec):
    import paper_1808_02515_gb300.sprintz as spz
    src = torch.arange(1000, dtype=torch.int32).to(torch.uint8).cuda()
    ptrs = torch.tensor([src.data_ptr(), src.data_ptr() + 100], dtype=torch.int64, device="cuda")
    sizes = torch.tensor([100, 200], dtype=torch.int64, device="cuda")
    dst = torch.full((299,), 7, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(3, dtype=torch.int64, device="cuda")
    codec.pack(ptrs, sizes, dst, offs)
    torch.cuda.synchronize()
    assert codec.status() == spz.ERR_DST_TOO_SMALL
    assert torch.all(dst == 7)
    assert offs.cpu().tolist() == [0, 100, 300]
