"""Wire form of ciphertext arrays (lc_wire_bytes / lc_pack / lc_unpack): byte layout against a
plain numpy packing written from the definition, round trips at toy and production size, and the
range check of unpack (GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(kind):
    from paper_2408_06197_b300 import lancelot as LC
    return LC, (LC.Context.toy() if kind == "toy" else LC.Context.production())


def _widths(q):
    return [min(8, max(4, (int(qi - 1).bit_length() + 7) // 8)) for qi in q]


def _np_pack(words, q, deg, level, N):
    """[count][deg][level+1][N] uint64 -> bytes: limb i's residues as w_i little-endian bytes."""
    w = _widths(q[:level + 1])
    recs = []
    for rec in words.reshape(-1, deg, level + 1, N):
        parts = []
        for p in range(deg):
            for i in range(level + 1):
                b = rec[p, i].astype("<u8").view(np.uint8).reshape(N, 8)[:, :w[i]]
                parts.append(b.reshape(-1))
        recs.append(np.concatenate(parts))
    return np.stack(recs)


def _residues(rng, q, shape_lead, level, N):
    return np.stack([rng.integers(0, qi, size=shape_lead + (N,), dtype=np.uint64) for qi in q[:level + 1]],
                    axis=-2)


@pytest.mark.parametrize("kind", ["toy", "prod"])
def test_pack_layout_and_round_trip(kind):
    LC, g = _ctx(kind)
    rng = np.random.default_rng(11)
    for deg, level, count in ((2, g.L, 3), (2, g.L - 1, 2), (3, g.L, 1)):
        words = _residues(rng, g.q, (count, deg), level, g.N)  # [count][deg][level+1][N]
        t = LC.u64_to_torch(np.ascontiguousarray(words))
        wire = g.pack(t, deg, level)
        assert wire.shape == (count, g.wire_bytes(deg, level))
        assert g.wire_bytes(deg, level) == deg * g.N * sum(_widths(g.q[:level + 1]))
        assert np.array_equal(wire.cpu().numpy(), _np_pack(words, g.q, deg, level, g.N))
        back = g.unpack(wire, count, deg, level)
        g.sync()
        assert np.array_equal(LC.torch_to_u64(back), words)
        # host-packed bytes unpack to the same words
        hw = torch.from_numpy(_np_pack(words, g.q, deg, level, g.N)).cuda()
        assert np.array_equal(LC.torch_to_u64(g.unpack(hw, count, deg, level)), words)
        g.sync()


def test_production_wire_size_and_range_check():
    LC, g = _ctx("prod")
    assert g.wire_bytes(2, g.L) == 2 * g.N * (8 + 14 * 5)  # 78 bytes per coefficient instead of 120
    rng = np.random.default_rng(12)
    words = _residues(rng, g.q, (1, 2), g.L, g.N)
    raw = _np_pack(words, g.q, 2, g.L, g.N)
    # residue 5 of limb 3 of polynomial 1 set to q_3 (not below its prime)
    w = _widths(g.q)
    off = g.N * sum(w[:g.L + 1]) + g.N * sum(w[:3]) + 5 * w[3]
    raw[0, off:off + w[3]] = np.frombuffer(int(g.q[3]).to_bytes(8, "little")[:w[3]], dtype=np.uint8)
    g.unpack(torch.from_numpy(raw).cuda(), 1, 2, g.L)
    with pytest.raises(LC.LancelotError, match="LC_EINVAL"):
        g.sync()
    good = torch.from_numpy(_np_pack(words, g.q, 2, g.L, g.N)).cuda()
    assert np.array_equal(LC.torch_to_u64(g.unpack(good, 1, 2, g.L)), words)
    g.sync()
