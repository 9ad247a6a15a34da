"""Pins of the oracle's byte-plane dictionary code and of the compressed
(version 2) image form, against constructed pages whose encodings follow
from the definition by hand, losslessness, canonical-form rejection and an
independent layout parser."""
from __future__ import annotations

import struct

import numpy as np
import pytest

import oracle
from oracle import bigint

P = 65536
N = 8192  # bytes per plane


def page_from_planes(planes):
    """65,536-byte slot whose plane j is planes[j] (8,192 bytes each)."""
    out = np.zeros(P, dtype=np.uint8)
    for j, pl in enumerate(planes):
        out[j::8] = pl
    return out


def test_zero_page_is_head_and_eight_padded_dicts():
    enc = oracle.bpd_encode(np.zeros(P, np.uint8))
    # every plane has k = 1 (b = 0): head 16 B + 8 x (1 dict byte padded to 16)
    assert len(enc) == 16 + 8 * 16
    assert enc == bytes(144)


def test_two_value_plane_packs_one_bit_per_byte_lsb_first():
    # plane 0 alternates 7, 200 (k = 2, b = 1): ranks 0,1,0,1,... -> bits
    # 0,1,0,1 from bit 0 of each byte -> every packed byte is 0b10101010
    planes = [np.zeros(N, np.uint8) for _ in range(8)]
    planes[0] = np.where(np.arange(N) % 2 == 0, 7, 200).astype(np.uint8)
    enc = oracle.bpd_encode(page_from_planes(planes))
    assert enc[0] == 1 and enc[8] == 1          # b = 1, k - 1 = 1
    assert enc[16:18] == bytes([7, 200])         # dictionary, ascending
    assert enc[18:32] == bytes(14)               # padding to 16
    assert enc[32:32 + 1024] == bytes([0xAA]) * 1024
    assert len(enc) == 16 + (16 + 1024) + 7 * 16


def test_three_value_plane_two_bits_per_index():
    # plane 3 cycles 9, 5, 250: dictionary [5, 9, 250], ranks 1, 0, 2, 1, 0, 2...
    planes = [np.zeros(N, np.uint8) for _ in range(8)]
    planes[3] = np.array([9, 5, 250], np.uint8)[np.arange(N) % 3]
    enc = oracle.bpd_encode(page_from_planes(planes))
    assert enc[3] == 2 and enc[11] == 2          # b = 2, k - 1 = 2
    base = 16 + 3 * 16                           # planes 0..2: one padded dict each
    assert enc[base:base + 3] == bytes([5, 9, 250])
    packed = enc[base + 16:base + 16 + 2048]
    ranks = [1, 0, 2]
    for i in (0, 1, 2, 3, 4, 5, 100, 8191):
        byte, shift = (2 * i) // 8, (2 * i) % 8
        assert (packed[byte] >> shift) & 3 == ranks[i % 3], i


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 16, 17, 64, 100, 128])
def test_length_follows_the_alphabet_size(k):
    rng = np.random.default_rng(k)
    planes = [np.zeros(N, np.uint8) for _ in range(8)]
    vals = np.sort(rng.choice(256, size=k, replace=False)).astype(np.uint8)
    planes[5] = vals[np.arange(N) % k]
    enc = oracle.bpd_encode(page_from_planes(planes))
    b = 0 if k == 1 else int(np.ceil(np.log2(k)))
    assert len(enc) == 16 + 7 * 16 + ((k + 15) // 16) * 16 + 1024 * b
    assert enc[5] == b and enc[13] == k - 1


def test_incompressible_slot_is_stored_as_is():
    slot = np.random.default_rng(3).integers(0, 256, P, dtype=np.uint8)
    enc = oracle.bpd_encode(slot)
    assert enc == slot.tobytes()


def test_mixed_raw_and_packed_planes():
    rng = np.random.default_rng(4)
    planes = [rng.integers(0, 256, N, dtype=np.uint8) for _ in range(8)]
    planes[7] = np.full(N, 0x3F, np.uint8)       # one value: b = 0
    planes[6] = rng.integers(0, 4, N, dtype=np.uint8) + 60  # 4 values: b = 2
    enc = oracle.bpd_encode(page_from_planes(planes))
    assert list(enc[:8]) == [8, 8, 8, 8, 8, 8, 2, 0]
    assert list(enc[8:16]) == [255] * 6 + [3, 0]
    assert len(enc) == 16 + 6 * N + (16 + 2048) + 16
    # a stored plane is the plane itself
    assert enc[16:16 + N] == planes[0].tobytes()


@pytest.mark.parametrize("seed", range(6))
def test_lossless_on_float_and_mixed_pages(seed):
    rng = np.random.default_rng(100 + seed)
    kind = seed % 3
    if kind == 0:
        slot = rng.uniform(-1, 1, P // 4).astype(np.float32).view(np.uint8)
    elif kind == 1:
        slot = rng.normal(size=P // 8).view(np.uint8)
    else:
        slot = page_from_planes([rng.integers(0, 1 << rng.integers(0, 9), N, dtype=np.uint64).astype(np.uint8)
                                 for _ in range(8)])
    enc = oracle.bpd_encode(slot)
    assert len(enc) % 16 == 0 and 16 <= len(enc) <= P
    st, dec = oracle.bpd_decode(enc)
    assert st == oracle.OK and dec == slot.tobytes()


def test_decoder_rejects_what_the_encoder_cannot_write():
    planes = [np.zeros(N, np.uint8) for _ in range(8)]
    planes[0] = np.array([1, 2, 3], np.uint8)[np.arange(N) % 3]
    enc = bytearray(oracle.bpd_encode(page_from_planes(planes)))
    assert oracle.bpd_decode(bytes(enc))[0] == oracle.OK
    bad = bytearray(enc); bad[0] = 3            # non-canonical width for k = 3
    assert oracle.bpd_decode(bytes(bad))[0] == oracle.CORRUPT
    bad = bytearray(enc); bad[16], bad[17] = 2, 1  # dictionary not ascending
    assert oracle.bpd_decode(bytes(bad))[0] == oracle.CORRUPT
    bad = bytearray(enc); bad[32] = 0xFF        # rank 3 >= k = 3
    assert oracle.bpd_decode(bytes(bad))[0] == oracle.CORRUPT
    assert oracle.bpd_decode(bytes(enc[:-16]))[0] == oracle.CORRUPT


def _parse_v2(img):
    magic, ver, flags, seq, parent, psz, A, n, poff, size = struct.unpack_from("<8sIIQQIIQQQ", img, 0)
    atab = [struct.unpack_from("<IIQ", img, 64 + 16 * a) for a in range(A)]
    base = 64 + 16 * A
    ptab = [struct.unpack_from("<II", img, base + 8 * s) for s in range(n)]
    hashes = [struct.unpack_from("<Q", img, base + 8 * n + 8 * s)[0] for s in range(n)]
    offs = [struct.unpack_from("<Q", img, base + 16 * n + 8 * s)[0] for s in range(n)]
    return dict(magic=magic, ver=ver, flags=flags, seq=seq, parent=parent, psz=psz, A=A, n=n,
                poff=poff, size=size, atab=atab, ptab=ptab, hashes=hashes, offs=offs)


def test_compressed_image_layout_and_restore():
    rng = np.random.default_rng(7)
    sizes = [3 * P + 100, P - 8, 5 * P]
    bufs = [rng.uniform(-1, 1, (n + 3) // 4).astype(np.float32).view(np.uint8)[:n].copy() for n in sizes]
    o = oracle.OracleSet(sizes, compress=True)
    img, d, h, _ = o.checkpoint(bufs)
    hd = _parse_v2(img)
    assert hd["magic"] == b"CRUMIMG1" and hd["ver"] == 2 and hd["flags"] == 3
    n = hd["n"]
    assert n == sum(-(-s // P) for s in sizes)
    assert hd["poff"] == (64 + 16 * hd["A"] + 24 * n + 15) // 16 * 16 and hd["size"] == len(img)
    assert hd["offs"][0] == 0 and all(b > a for a, b in zip(hd["offs"], hd["offs"][1:]))
    assert hd["hashes"] == [int(x) for x in h]
    # trailer by the independent big-integer hash
    assert struct.unpack_from("<Q", img, len(img) - 8)[0] == bigint.hash_bytes(img[:-8], 0)
    # every slot decodes to the page's valid bytes then zeros
    total = len(img) - 8 - hd["poff"]
    ends = hd["offs"][1:] + [total]
    g = 0
    for a, n_bytes in enumerate(sizes):
        for p in range(-(-n_bytes // P)):
            enc = img[hd["poff"] + hd["offs"][g]:hd["poff"] + ends[g]]
            st, slot = oracle.bpd_decode(enc)
            valid = min(P, n_bytes - p * P)
            want = bufs[a][p * P:p * P + valid].tobytes() + bytes(P - valid)
            assert st == oracle.OK and slot == want
            g += 1
    assert len(img) < oracle.image_size(len(sizes), n)  # float pages do shrink
    # restore onto garbage
    garbage = [np.full(s, 0xCD, np.uint8) for s in sizes]
    hp = np.zeros(n, np.uint64)
    assert oracle.apply_image(img, garbage, hp) == oracle.OK
    assert all(np.array_equal(g_, b_) for g_, b_ in zip(garbage, bufs))
    assert np.array_equal(hp, h)
    # corruption is detected
    bad = bytearray(img); bad[hd["poff"] + 20] ^= 1
    assert oracle.check_image(bytes(bad)) == oracle.CORRUPT


def test_compressed_chain_replays_like_the_uncompressed_one():
    rng = np.random.default_rng(8)
    sizes = [4 * P + 24, 2 * P]
    bufs = [rng.normal(size=(n + 7) // 8).view(np.uint8)[:n].copy() for n in sizes]
    oc, ou = oracle.OracleSet(sizes, compress=True), oracle.OracleSet(sizes)
    chain_c, chain_u, states = [], [], []
    for step in range(3):
        if step:
            for b in bufs:
                b[rng.integers(0, b.size, 200)] ^= 0x5A
        chain_c.append(oc.checkpoint(bufs)[0])
        chain_u.append(ou.checkpoint(bufs)[0])
        states.append([b.copy() for b in bufs])
    for k in range(3):
        out_c = [np.zeros(s, np.uint8) for s in sizes]
        out_u = [np.zeros(s, np.uint8) for s in sizes]
        assert oracle.OracleSet(sizes).restore(chain_c[:k + 1], out_c) == oracle.OK
        assert oracle.OracleSet(sizes).restore(chain_u[:k + 1], out_u) == oracle.OK
        assert all(np.array_equal(a, b) for a, b in zip(out_c, states[k]))
        assert all(np.array_equal(a, b) for a, b in zip(out_u, states[k]))
