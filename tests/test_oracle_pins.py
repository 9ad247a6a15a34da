"""Pins for the CPU oracle: published values, closed forms, invariants and
brute force, so that a mistake anywhere in the oracle (a wrong constant or
shift, a dropped index term, a wrong padding rule, a transposed table) fails
here without reference to the oracle itself."""
import random
import struct

import numpy as np
import pytest

import oracle
from oracle import bigint as B

M64 = (1 << 64) - 1
PHI = 0x9E3779B97F4A7C15


# ---- the mixer against the published splitmix64 sequences ----

def test_bigint_generator_matches_published(published_splitmix64):
    for seed, outs in published_splitmix64.items():
        assert B.splitmix64(seed, len(outs)) == outs


def test_c_mix_matches_published(published_splitmix64):
    # output k of the generator seeded with s is mix(s + k*phi)
    for seed, outs in published_splitmix64.items():
        for k, v in enumerate(outs, start=1):
            assert oracle.mix((seed + k * PHI) & M64) == v


def test_mix_zero_is_zero():
    # closed form: every step of mix maps 0 to 0
    assert oracle.mix(0) == 0 and B.mix(0) == 0


def test_mix_is_a_bijection():
    # unmix is built from the algebra (xorshift undo, modular inverses);
    # it inverts the C mix exactly, so mix is one-to-one on 64-bit words
    rng = random.Random(7)
    for _ in range(2000):
        x = rng.getrandbits(64)
        assert B.unmix(oracle.mix(x)) == x


# ---- the page hash against the published sequences ----

def test_single_word_page_is_one_generator_output(published_splitmix64):
    # a page of one word w hashes to mix(w XOR 0) = mix(w)
    for seed, outs in published_splitmix64.items():
        w = (seed + PHI) & M64
        assert oracle.page_hash(struct.pack("<Q", w)) == outs[0]


def test_constructed_page_sums_published_outputs(published_splitmix64):
    # word 0 = 0 contributes mix(0) = 0; word i = (s + i*phi) XOR (i*phi)
    # contributes mix(s + i*phi) = output i of the generator seeded with s.
    for seed, outs in published_splitmix64.items():
        ws = [0] + [((seed + i * PHI) & M64) ^ ((i * PHI) & M64) for i in range(1, len(outs) + 1)]
        buf = b"".join(struct.pack("<Q", w) for w in ws)
        assert oracle.page_hash(buf) == sum(outs) & M64
        assert B.hash_bytes(buf) == sum(outs) & M64


def test_zero_words_sum_seed0_outputs(published_splitmix64):
    outs = published_splitmix64[0]
    for n in range(1, len(outs) + 2):
        assert oracle.page_hash(b"\0" * (8 * n)) == sum(outs[: n - 1]) & M64
    assert oracle.page_hash(b"\0" * 24) == 0x509946A41CD733A3


# ---- C oracle vs the independent big-integer rendering on tiny inputs ----

def _patterns():
    rng = random.Random(11)
    out = []
    for n in [1, 2, 7, 8, 9, 15, 16, 17, 23, 24, 31, 33, 40, 64, 100, 255]:
        out.append(b"\0" * n)
        out.append(b"\xff" * n)
        out.append(bytes(rng.getrandbits(8) for _ in range(n)))
        ws = b"".join(struct.pack("<Q", i) for i in range((n + 7) // 8))[:n]
        out.append(ws)
        one_bit = bytearray(n)
        one_bit[rng.randrange(n)] = 1 << rng.randrange(8)
        out.append(bytes(one_bit))
    return out


@pytest.mark.parametrize("first", [0, 1, 8191, 2**40 + 3])
def test_c_hash_equals_bigint(first):
    for buf in _patterns():
        assert oracle.hash_bytes(buf, first) == B.hash_bytes(buf, first)


def test_partial_word_is_zero_padded_and_no_extra_words():
    rng = random.Random(3)
    for n in range(1, 64):
        buf = bytes(rng.getrandbits(8) for _ in range(n))
        padded = buf + b"\0" * ((-n) % 8)
        assert oracle.page_hash(buf) == oracle.page_hash(padded)
        # a further all-zero word is a real word: it adds mix(nw * phi) != 0
        nw = len(padded) // 8
        assert oracle.page_hash(padded + b"\0" * 8) == (oracle.page_hash(padded) + B.mix(nw * PHI)) & M64


def test_tree_reducible():
    rng = np.random.default_rng(5)
    buf = rng.integers(0, 256, size=65536, dtype=np.uint8).tobytes()
    whole = oracle.page_hash(buf)
    for cut_words in [1, 17, 4096, 8191]:
        a = oracle.hash_bytes(buf[: 8 * cut_words], 0)
        b = oracle.hash_bytes(buf[8 * cut_words:], cut_words)
        assert (a + b) & M64 == whole
    # any order of per-word terms: shuffle the words, keep each index
    words = np.frombuffer(buf, dtype=np.uint64)
    perm = rng.permutation(words.size)
    terms = [oracle.hash_bytes(words[i:i + 1].tobytes(), int(i)) for i in perm[:512]]
    rest = sorted(set(range(words.size)) - set(int(i) for i in perm[:512]))
    s = sum(terms) + sum(oracle.hash_bytes(words[i:i + 1].tobytes(), i) for i in rest)
    assert s & M64 == whole


def test_every_single_word_change_is_detected():
    # brute force on a small page: every word position, many new values
    rng = np.random.default_rng(9)
    words = rng.integers(0, 2**63, size=64, dtype=np.uint64)
    base = oracle.page_hash(words.tobytes())
    for i in range(words.size):
        for delta in [1, 1 << 63, 0xFFFFFFFFFFFFFFFF] + [int(x) | 1 for x in rng.integers(0, 2**63, size=8)]:
            w = words.copy()
            w[i] ^= np.uint64(delta)
            assert oracle.page_hash(w.tobytes()) != base


def test_every_single_byte_value_is_detected():
    # exhaustive over one byte position per word of a 4-word page
    buf = bytearray(32)
    base = oracle.page_hash(bytes(buf))
    for pos in range(32):
        for v in range(1, 256):
            b = bytearray(buf)
            b[pos] = v
            assert oracle.page_hash(bytes(b)) != base


# ---- page geometry ----

def test_page_geometry():
    P = oracle.PAGE
    assert oracle.pages_of(1) == 1 and oracle.pages_of(P) == 1 and oracle.pages_of(P + 1) == 2
    assert oracle.valid_bytes(P + 1, 1) == 1 and oracle.valid_bytes(3 * P, 2) == P
    assert oracle.total_pages([P, 1, 4 * P + 8]) == 1 + 1 + 5


def test_hash_all_matches_per_page_bigint():
    rng = np.random.default_rng(1)
    sizes = [8, 4096 + 3, 65536, 65536 + 24, 3 * 65536 - 5]
    allocs = [rng.integers(0, 256, size=s, dtype=np.uint8) for s in sizes]
    got = oracle.hash_all(allocs)
    exp = []
    for a in allocs:
        b = a.tobytes()
        for p in range(0, len(b), 65536):
            exp.append(B.hash_bytes(b[p:p + 65536]))
    assert [int(x) for x in got] == exp


# ---- dirty rule ----

def test_dirty_rule():
    h = np.array([1, 2, 3, 4], dtype=np.uint64)
    hp = np.array([1, 9, 3, 4], dtype=np.uint64)
    d, n = oracle.dirty(h, hp, None, False)
    assert list(d) == [0, 1, 0, 0] and n == 1
    d, n = oracle.dirty(h, hp, np.array([0, 0, 0, 1], np.uint8), False)
    assert list(d) == [0, 1, 0, 1] and n == 2
    d, n = oracle.dirty(h, hp, None, True)
    assert list(d) == [1, 1, 1, 1] and n == 4


# ---- image format, parsed independently ----

def _parse(img: bytes):
    magic, ver, flags, seq, parent, psz, A, n, poff, size = struct.unpack_from("<8sIIQQIIQQQ", img, 0)
    allocs = [struct.unpack_from("<IIQ", img, 64 + 16 * a) for a in range(A)]
    ptab = [struct.unpack_from("<II", img, 64 + 16 * A + 8 * s) for s in range(n)]
    hashes = [struct.unpack_from("<Q", img, 64 + 16 * A + 8 * n + 8 * s)[0] for s in range(n)]
    payload = [img[poff + 65536 * s: poff + 65536 * (s + 1)] for s in range(n)]
    trailer = struct.unpack_from("<Q", img, len(img) - 8)[0]
    return dict(magic=magic, ver=ver, flags=flags, seq=seq, parent=parent, psz=psz, A=A, n=n,
                poff=poff, size=size, allocs=allocs, ptab=ptab, hashes=hashes, payload=payload,
                trailer=trailer)


def test_image_layout_independent_parse():
    rng = np.random.default_rng(2)
    sizes = [65536 * 2 + 100, 4096]
    allocs = [rng.integers(0, 256, size=s, dtype=np.uint8) for s in sizes]
    h = oracle.hash_all(allocs)
    d = np.array([0, 1, 1, 1], dtype=np.uint8)
    img = oracle.build_image(allocs, [5, 9], h, d, False, 7, 6)
    p = _parse(img)
    assert p["magic"] == b"CRUMIMG1" and p["ver"] == 1 and p["flags"] == 0
    assert (p["seq"], p["parent"], p["psz"], p["A"], p["n"]) == (7, 6, 65536, 2, 3)
    assert p["poff"] == 64 + 32 + 48 and p["size"] == len(img) == p["poff"] + 3 * 65536 + 8
    assert p["allocs"] == [(5, 0, sizes[0]), (9, 0, sizes[1])]
    assert p["ptab"] == [(0, 1), (0, 2), (1, 0)]
    assert p["hashes"] == [int(h[1]), int(h[2]), int(h[3])]
    a0 = allocs[0].tobytes()
    assert p["payload"][0] == a0[65536:131072]
    assert p["payload"][1] == a0[131072:] + b"\0" * (65536 - 100)
    assert p["payload"][2] == allocs[1].tobytes() + b"\0" * (65536 - 4096)
    # each stored hash is the big-integer hash of that page's valid bytes
    assert p["hashes"][1] == B.hash_bytes(a0[131072:])
    # trailer: the hash over every preceding byte, computed independently
    assert p["trailer"] == B.hash_bytes(img[:-8])
    assert oracle.check_image(img) == oracle.OK


def test_full_image_has_no_parent():
    a = np.zeros(10, dtype=np.uint8)
    img = oracle.build_image([a], [0], oracle.hash_all([a]), np.ones(1, np.uint8), True, 0, 123)
    p = _parse(img)
    assert p["flags"] == 1 and p["parent"] == 0xFFFFFFFFFFFFFFFF


def test_corruption_and_truncation_detected():
    rng = np.random.default_rng(4)
    a = rng.integers(0, 256, size=70000, dtype=np.uint8)
    s = oracle.OracleSet([a.size])
    img, *_ = s.checkpoint([a])
    assert oracle.check_image(img) == oracle.OK
    for pos in [0, 9, 40, 64, 72, 80, len(img) // 2, len(img) - 1]:
        b = bytearray(img)
        b[pos] ^= 0x10
        assert oracle.check_image(bytes(b)) == oracle.CORRUPT
    assert oracle.check_image(img[:-1]) == oracle.CORRUPT
    assert oracle.check_image(img[: len(img) // 2]) == oracle.CORRUPT


# ---- checkpoint / restore invariants ----

def _mutate(allocs, rng, frac):
    """xor a nonzero mask into one random word of chosen pages; returns the
    set of global pages touched."""
    touched, g0 = set(), 0
    for a in allocs:
        n = oracle.pages_of(a.size)
        for p in range(n):
            if rng.random() < frac:
                v = oracle.valid_bytes(a.size, p)
                pos = p * 65536 + int(rng.integers(0, v))
                a[pos] ^= np.uint8(int(rng.integers(1, 256)))
                touched.add(g0 + p)
        g0 += n
    return touched


def test_checkpoint_restore_chain_roundtrip():
    rng = np.random.default_rng(6)
    sizes = [3 * 65536 + 5, 65536, 4096 + 8, 200000]
    allocs = [rng.integers(0, 256, size=s, dtype=np.uint8) for s in sizes]
    s = oracle.OracleSet(sizes)
    img0, d0, h0, _ = s.checkpoint(allocs)
    assert d0.all() and _parse(img0)["flags"] == 1
    chain, states = [img0], [[a.copy() for a in allocs]]
    for step in range(5):
        touched = _mutate(allocs, rng, 0.3)
        img, d, h, _ = s.checkpoint(allocs)
        # dirty set equals exactly the mutated set
        assert set(np.nonzero(d)[0].tolist()) == touched
        p = _parse(img)
        assert p["parent"] == step and p["seq"] == step + 1 and p["n"] == len(touched)
        chain.append(img)
        states.append([a.copy() for a in allocs])
    # unchanged state: empty incremental
    img_e, d_e, _, _ = s.checkpoint(allocs)
    assert d_e.sum() == 0 and _parse(img_e)["n"] == 0
    # replay each prefix of the chain onto garbage: equals that step's state
    for k in range(len(chain)):
        garbage = [rng.integers(0, 256, size=sz, dtype=np.uint8) for sz in sizes]
        r = oracle.OracleSet(sizes)
        assert r.restore(chain[: k + 1], garbage) == oracle.OK
        for got, exp in zip(garbage, states[k]):
            assert np.array_equal(got, exp)
        # restored hash table equals the hashes of the restored state
        assert np.array_equal(r.h_prev, oracle.hash_all(states[k]))
        # next checkpoint of the restored set is empty and has the right parent
        img_n, d_n, _, _ = r.checkpoint(garbage)
        assert d_n.sum() == 0 and _parse(img_n)["parent"] == k


def test_registration_change_starts_a_new_full_chain():
    """Algorithm 1: a region that starts being tracked has every page dirty.
    After register or unregister the next image is full (no parent, every
    page of every registered allocation, ids as assigned), sequence numbers
    keep counting, and the next image after that is an ordinary incremental
    of the new table.  Checked with the independent struct parser, the
    big-integer hash and a restore of the new chain onto garbage."""
    rng = np.random.default_rng(8)
    sizes = [2 * 65536 + 12, 65536]
    allocs = [rng.integers(0, 256, size=s, dtype=np.uint8) for s in sizes]
    s = oracle.OracleSet(sizes)
    s.checkpoint(allocs)
    _mutate(allocs, rng, 0.5)
    s.checkpoint(allocs)
    extra = rng.integers(0, 256, size=3 * 65536 + 4096, dtype=np.uint8)
    assert s.register(extra.size) == 2
    allocs3 = allocs + [extra]
    img, d, h, _ = s.checkpoint(allocs3)
    p = _parse(img)
    assert p["flags"] == 1 and p["seq"] == 2 and p["parent"] == 0xFFFFFFFFFFFFFFFF
    assert d.all() and p["n"] == 3 + 1 + 4
    assert p["allocs"] == [(0, 0, sizes[0]), (1, 0, sizes[1]), (2, 0, extra.size)]
    assert p["ptab"] == [(0, 0), (0, 1), (0, 2), (1, 0), (2, 0), (2, 1), (2, 2), (2, 3)]
    assert p["hashes"][5] == B.hash_bytes(extra[65536:131072].tobytes())
    assert p["payload"][7] == extra[3 * 65536:].tobytes() + b"\0" * (65536 - 4096)
    assert p["trailer"] == B.hash_bytes(img[:-8])
    # the next image is incremental again, parented on the new base
    touched = _mutate(allocs3, rng, 0.4)
    img2, d2, _, _ = s.checkpoint(allocs3)
    p2 = _parse(img2)
    assert p2["flags"] == 0 and p2["seq"] == 3 and p2["parent"] == 2
    assert set(np.nonzero(d2)[0].tolist()) == touched
    # unregistering the first allocation: ids 1 and 2 stay, a full image again
    s.unregister(0)
    img3, d3, _, _ = s.checkpoint(allocs3[1:])
    p3 = _parse(img3)
    assert p3["flags"] == 1 and p3["seq"] == 4 and p3["parent"] == 0xFFFFFFFFFFFFFFFF
    assert p3["allocs"] == [(1, 0, sizes[1]), (2, 0, extra.size)] and d3.all() and p3["n"] == 5
    assert p3["ptab"][0] == (0, 0) and p3["ptab"][1] == (1, 0)
    assert p3["payload"][0] == allocs[1].tobytes()
    assert p3["trailer"] == B.hash_bytes(img3[:-8])
    # the chain that began at the registration change restores onto garbage
    garbage = [rng.integers(0, 256, size=a.size, dtype=np.uint8) for a in allocs3]
    r = oracle.OracleSet([a.size for a in allocs3])
    assert r.restore([img, img2], garbage) == oracle.OK
    for got, exp in zip(garbage, allocs3):
        assert np.array_equal(got, exp)


def test_restore_mismatch():
    a = np.zeros(70000, dtype=np.uint8)
    img, *_ = oracle.OracleSet([a.size]).checkpoint([a])
    b = np.zeros(70001, dtype=np.uint8)
    assert oracle.apply_image(img, [b], None) == oracle.MISMATCH
    assert oracle.apply_image(img, [a, b], None) == oracle.MISMATCH


def test_verify_mode_catches_injected_collision():
    rng = np.random.default_rng(8)
    a = rng.integers(0, 256, size=4 * 65536, dtype=np.uint8)
    s = oracle.OracleSet([a.size])
    s.checkpoint([a])
    prev = a.copy()
    a[2 * 65536 + 10] ^= 0xFF
    # inject: make the stored hash of page 2 equal the new hash, so the
    # hash alone calls the changed page clean
    s.h_prev[2] = oracle.hash_all([a])[2]
    img, d, h, coll = s.checkpoint([a], verify_prev=[prev])
    assert coll == 1 and d[2] == 1 and _parse(img)["ptab"] == [(0, 2)]
    # without verify mode the collision goes unseen
    s2 = oracle.OracleSet([a.size])
    s2.checkpoint([prev])
    s2.h_prev[2] = oracle.hash_all([a])[2]
    _, d2, _, _ = s2.checkpoint([a])
    assert d2.sum() == 0
