"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: brute force over all
permutations of tiny inputs, the invariants that characterise a stable sort,
closed-form special cases, hand-built examples of Alg. 2's bucket numbering
and heavy-key rule, the published SplitMix64 outputs, and Alg. 3's output on
random zones.  ``test_planted_mistakes_are_caught`` rebuilds oracle.c with a
plausible bug planted and checks that these pins fail on it.
"""
import itertools
import os
import subprocess

import numpy as np
import pytest

import gen
import oracle

W32 = np.uint32
W64 = np.uint64


# ---------------------------------------------------------------- brute force
def brute_force_stable(keys):
    """The unique permutation pi with keys[pi] non-decreasing and, among equal
    keys, pi increasing -- found by enumerating every permutation."""
    n = len(keys)
    found = []
    for perm in itertools.permutations(range(n)):
        ok = True
        for a, b in zip(perm, perm[1:]):
            if keys[a] > keys[b] or (keys[a] == keys[b] and a > b):
                ok = False
                break
        if ok:
            found.append(perm)
    assert len(found) == 1
    return np.array(found[0], dtype=np.int64)


@pytest.mark.parametrize("dtype", [W32, W64])
def test_brute_force_all_small_inputs(dtype):
    top = int(np.iinfo(dtype).max)
    alphabet = [0, 1, 2, top]
    for n in range(0, 6):
        for combo in itertools.product(alphabet, repeat=n):
            keys = np.array(combo, dtype=dtype)
            vals = np.arange(n, dtype=dtype)
            ok, ov = oracle.stable_sort(keys, vals)
            if n == 0:
                assert len(ok) == 0
                continue
            pi = brute_force_stable(list(combo))
            np.testing.assert_array_equal(ok, keys[pi])
            np.testing.assert_array_equal(ov, vals[pi])


def test_brute_force_length6_sampled():
    rs = np.random.RandomState(7)
    alphabet = np.array([0, 1, 2, 2**32 - 1], dtype=W32)
    for _ in range(120):
        keys = alphabet[rs.randint(0, 4, size=6)]
        vals = (np.arange(6) * 7 + 3).astype(W32)
        ok, ov = oracle.stable_sort(keys, vals)
        pi = brute_force_stable(list(keys))
        np.testing.assert_array_equal(ok, keys[pi])
        np.testing.assert_array_equal(ov, vals[pi])


# ----------------------------------------------------------------- invariants
def check_stable_sort(keys, vals_idx, ok, ov):
    """Sortedness, stability (values = original index increase inside runs of
    equal keys), permutation (index bitmap, key agreement, multiset hash and
    per-top-16-bit counts).  Together these fix the output uniquely."""
    n = len(keys)
    assert len(ok) == n and len(ov) == n
    if n == 0:
        return
    assert np.all(ok[1:] >= ok[:-1]), "not sorted"
    idx = ov.astype(np.int64)
    seen = np.zeros(n, dtype=bool)
    assert idx.min() >= 0 and idx.max() < n
    seen[idx] = True
    assert seen.all(), "values are not a permutation of the indices"
    np.testing.assert_array_equal(keys[idx], ok)
    same = ok[1:] == ok[:-1]
    assert np.all(idx[1:][same] > idx[:-1][same]), "not stable"
    shift = 48 if keys.dtype == W64 else 16
    np.testing.assert_array_equal(
        np.bincount((keys >> shift).astype(np.int64), minlength=65536),
        np.bincount((ok >> shift).astype(np.int64), minlength=65536))

    def mh(k, v):
        with np.errstate(over="ignore"):
            x = (k.astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)) ^ v.astype(np.uint64)
            x ^= x >> np.uint64(29)
            x *= np.uint64(0xBF58476D1CE4E5B9)
            return int(x.sum(dtype=np.uint64))
    assert mh(keys, vals_idx) == mh(ok, ov)


@pytest.mark.parametrize("name", sorted(gen.U32_FAMILIES))
def test_invariants_u32_families(name):
    n = 200_003
    keys = gen.family(name, n, W32, seed=3)
    vals = gen.iota(n, W32)
    ok, ov = oracle.stable_sort(keys, vals, nthreads=4)
    check_stable_sort(keys, vals, ok, ov)


@pytest.mark.parametrize("name", sorted(gen.U64_FAMILIES))
def test_invariants_u64_families(name):
    n = 100_001
    keys = gen.family(name, n, W64, seed=5)
    vals = gen.iota(n, W64)
    ok, ov = oracle.stable_sort(keys, vals, nthreads=3)
    check_stable_sort(keys, vals, ok, ov)


def test_second_formulation_numpy_stable_argsort():
    # an independent formulation (numpy's stable sort of the keys alone)
    for dtype in (W32, W64):
        keys = gen.family("zipf1.2hash", 300_000, dtype, seed=11)
        vals = gen.iota(len(keys), dtype)
        ok, ov = oracle.stable_sort(keys, vals, nthreads=5)
        p = np.argsort(keys, kind="stable")
        np.testing.assert_array_equal(ok, keys[p])
        np.testing.assert_array_equal(ov, vals[p])


def test_thread_count_does_not_change_output():
    keys = gen.family("bitexp", 100_000, W32, seed=2)
    vals = gen.iota(len(keys), W32)
    ref = oracle.stable_sort(keys, vals, nthreads=1)
    for t in (2, 3, 7, 16):
        out = oracle.stable_sort(keys, vals, nthreads=t)
        np.testing.assert_array_equal(out[0], ref[0])
        np.testing.assert_array_equal(out[1], ref[1])


def test_key_only_matches_key_value_keys():
    keys = gen.family("zipf1.0", 50_000, W32, seed=9)
    ok, ov = oracle.stable_sort(keys)
    assert ov is None
    ok2, _ = oracle.stable_sort(keys, gen.iota(len(keys), W32))
    np.testing.assert_array_equal(ok, ok2)


# --------------------------------------------------------------- closed forms
def test_all_equal_is_identity():
    for dtype in (W32, W64):
        keys = np.full(10_000, 12345, dtype=dtype)
        vals = gen.iota(10_000, dtype)
        ok, ov = oracle.stable_sort(keys, vals)
        np.testing.assert_array_equal(ov, vals)
        np.testing.assert_array_equal(ok, keys)


def test_sorted_input_is_identity_and_reverse_reverses():
    keys = np.arange(0, 3 * 50_000, 3, dtype=W32)
    vals = gen.iota(len(keys), W32)
    ok, ov = oracle.stable_sort(keys, vals)
    np.testing.assert_array_equal(ov, vals)
    ok, ov = oracle.stable_sort(keys[::-1].copy(), vals)
    np.testing.assert_array_equal(ov, vals[::-1])


def test_ten_distinct_keys_run_lengths():
    n = 100_000
    keys = gen.family("distinct10", n, W32, seed=4)
    vals = gen.iota(n, W32)
    ok, ov = oracle.stable_sort(keys, vals)
    uniq, counts = np.unique(keys, return_counts=True)
    assert len(uniq) == 10
    # runs appear in key order with lengths equal to the input counts, and
    # inside a run the original indices are exactly the ones holding that key
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    for u, c, s in zip(uniq, counts, starts):
        assert np.all(ok[s:s + c] == u)
        np.testing.assert_array_equal(ov[s:s + c], np.nonzero(keys == u)[0])


def test_extreme_keys():
    for dtype in (W32, W64):
        top = np.iinfo(dtype).max
        keys = np.array([top, 0, top, 1, 0, top - 1], dtype=dtype)
        ok, ov = oracle.stable_sort(keys, np.arange(6, dtype=dtype))
        np.testing.assert_array_equal(ok, [0, 0, 1, top - 1, top, top])
        np.testing.assert_array_equal(ov, [1, 4, 3, 5, 0, 2])


# ------------------------------------------------------------------ segmented
def test_segmented_is_per_segment():
    rs = np.random.RandomState(1)
    sizes = rs.randint(0, 700, size=60)
    sizes[[3, 10, 11]] = 0
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    keys = gen.family("zipf1.0", n, W32, seed=5)
    vals = gen.iota(n, W32)
    ok, ov = oracle.stable_sort_segmented(keys, vals, off)
    for s in range(len(sizes)):
        a, b = off[s], off[s + 1]
        seg_k = keys[a:b]
        p = brute_order(seg_k)
        np.testing.assert_array_equal(ok[a:b], seg_k[p])
        np.testing.assert_array_equal(ov[a:b], vals[a:b][p])


def brute_order(k):
    # stable order by definition, via Python's sort on (key, index) tuples
    return np.array(sorted(range(len(k)), key=lambda i: (int(k[i]), i)),
                    dtype=np.int64)


# ------------------------------------------------------------ stable positions
def test_stable_positions_match_definition():
    rs = np.random.RandomState(3)
    keys = rs.randint(0, 20, size=500).astype(W32)
    js = np.arange(500)
    pos = oracle.stable_positions(keys, js, nthreads=3)
    p = brute_order(keys)
    inv = np.empty(500, dtype=np.int64)
    inv[p] = np.arange(500)
    np.testing.assert_array_equal(pos, inv)


# --------------------------------------------------------------------- RNG
def test_splitmix64_published_values():
    # SplitMix64 from state 0 (Steele, Lea, Flood 2014 reference generator)
    assert oracle.splitmix64_sequence(0, 3) == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # the counter form: output i from state s equals the i-th sequential output
    seq = oracle.splitmix64_sequence(12345, 5)
    assert [oracle.splitmix64_at(12345, i) for i in range(5)] == seq


def test_sample_positions_in_range_and_deterministic():
    p1 = oracle.sample_positions(7, 1000, 333, 32, 5000)
    p2 = oracle.sample_positions(7, 1000, 333, 32, 5000)
    np.testing.assert_array_equal(p1, p2)
    assert p1.min() >= 1000 and p1.max() < 1333
    # every position of a small range is hit (uniform draws, 5000 >> 333)
    assert len(np.unique(p1)) == 333
    p3 = oracle.sample_positions(7, 1000, 333, 31, 5000)
    assert not np.array_equal(p1, p3)


# --------------------------------------------------------- heavy-key rule (Alg. 2)
def test_heavy_rule_hand_example():
    # sorted S (m = 15), stride L = 3: S' = S[2], S[5], S[8], S[11], S[14]
    S = [1, 1, 1, 1, 1, 1, 2, 3, 3, 3, 3, 3, 3, 4, 5]
    rs = np.random.RandomState(0)
    shuffled = np.array(S, dtype=np.uint64)[rs.permutation(15)]
    heavy, mx = oracle.heavy_from_sample(shuffled, 3)
    # S' = [1, 1, 3, 3, 5]
    np.testing.assert_array_equal(heavy, [1, 3])
    assert mx == 5
    # a run of length L that covers only one subsample point is not heavy
    S2 = [0, 7, 7, 7, 9, 9]          # S' = S[2], S[5] = [7, 9]
    heavy, _ = oracle.heavy_from_sample(np.array(S2, dtype=np.uint64), 3)
    assert len(heavy) == 0
    # a run of length L+1 starting at a subsample point covers two of them
    S3 = [4, 4, 5, 5, 5, 5, 6, 6, 6]  # S' = S[2], S[5], S[8] = [5, 5, 6]
    heavy, _ = oracle.heavy_from_sample(np.array(S3, dtype=np.uint64), 3)
    np.testing.assert_array_equal(heavy, [5])


def test_heavy_rule_against_run_positions():
    # heavy <=> the key's run [first, last] in sorted S contains at least two
    # of the positions L-1, 2L-1, ... (< m): checked on random samples
    rs = np.random.RandomState(5)
    for _ in range(300):
        m = rs.randint(1, 200)
        L = rs.randint(1, 12)
        S = rs.zipf(1.6, size=m).astype(np.uint64)
        heavy, mx = oracle.heavy_from_sample(S, L)
        s = np.sort(S)
        expect = []
        for key in np.unique(s):
            first = np.searchsorted(s, key, "left")
            last = np.searchsorted(s, key, "right") - 1
            pts = [p for p in range(L - 1, (m // L) * L, L) if first <= p <= last]
            if len(pts) >= 2:
                expect.append(key)
        np.testing.assert_array_equal(heavy, np.array(expect, dtype=np.uint64))
        assert mx == s[-1]


def test_ten_distinct_keys_all_heavy_at_root():
    # Thm 3.5: with at most c' 2^gamma distinct keys every key is heavy whp.
    n = 1_000_000
    keys = gen.family("distinct10", n, W32, seed=1)
    L = int(np.ceil(np.log2(n)))
    gamma = 8
    heavy, _ = oracle.sample_heavy(keys, 1, 0, n, 32, (1 << gamma) * L, L)
    np.testing.assert_array_equal(heavy, np.unique(keys).astype(np.uint64))


def test_uniform_keys_have_no_heavy():
    n = 1_000_000
    keys = gen.family("uniform", n, W32, seed=1)
    L = 20
    heavy, mx = oracle.sample_heavy(keys, 1, 0, n, 32, 256 * L, L)
    assert len(heavy) == 0
    assert mx >= 2**31


def test_heavy_threshold_statistics():
    # a key with frequency well above 1/|S'| is detected, one well below not:
    # 5% of records = key A (>> 1/256), 0.05% = key B (<< 1/256)
    n = 400_000
    rs = np.random.RandomState(2)
    keys = rs.randint(0, 2**32 - 1, size=n, dtype=np.uint64).astype(W32)
    keys[rs.rand(n) < 0.05] = 77
    keys[rs.rand(n) < 0.0005] = 99
    L = 19
    hits_a = hits_b = 0
    for seed in range(20):
        heavy, _ = oracle.sample_heavy(keys, seed, 0, n, 32, 256 * L, L)
        hits_a += 77 in heavy
        hits_b += 99 in heavy
    assert hits_a == 20 and hits_b == 0


# ------------------------------------------------------ bucket numbering (Alg. 2)
def test_bucket_ids_hand_example_r16_gamma2():
    # r = 16 (hi = 4 bits), gamma = 2, largest sample 15 -> zones are bits [2,4)
    # heavy {5, 6, 13}: zone 0 light 0; zone 1 light 1, 5 -> 2, 6 -> 3;
    # zone 2 light 4; zone 3 light 5, 13 -> 6; overflow 7
    keys = np.arange(16, dtype=W32)
    ids, nb = oracle.bucket_ids([13, 5, 6], 15, 4, 2, keys)
    np.testing.assert_array_equal(
        ids, [0, 0, 0, 0, 1, 2, 3, 1, 4, 4, 4, 4, 5, 6, 5, 5])
    assert nb == 8
    # largest sample 7: t = 3, zones are bits [1, 3); keys >= 8 overflow
    ids, nb = oracle.bucket_ids([5, 6], 7, 4, 2, keys)
    np.testing.assert_array_equal(
        ids, [0, 0, 1, 1, 2, 3, 5, 4, 6, 6, 6, 6, 6, 6, 6, 6])
    assert nb == 7


def _golden(name):
    """A text fixture under tests/golden: '#' comments, then 'field v1 v2 ...'
    lines; returns {field: [int, ...]}."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    out = {}
    for line in open(path):
        line = line.split("#", 1)[0].split()
        if line:
            out[line[0]] = [int(v) for v in line[1:]]
    return out


def test_golden_overflow_bucket_example():
    # the paper's overflow-bucket example (see the fixture's header): two key
    # bits, largest sampled key 1 -> zones 00 and 01, keys 10 and 11 overflow
    g = _golden("overflow_bucket_two_bits.txt")
    keys = np.array(g["keys"], dtype=W32)
    for gamma in g["gamma"]:
        assert oracle.zone_layout(g["sample_max"][0], g["hi"][0], gamma) == tuple(g["zone_bits"])
        ids, nb = oracle.bucket_ids([], g["sample_max"][0], g["hi"][0], gamma, keys)
        np.testing.assert_array_equal(ids, g["ids"])
        assert nb == g["buckets"][0]


def test_zone_layout():
    assert oracle.zone_layout(15, 4, 2) == (4, 2)
    assert oracle.zone_layout(7, 4, 2) == (3, 1)
    assert oracle.zone_layout(1, 32, 8) == (1, 0)
    assert oracle.zone_layout(0, 32, 8) == (0, 0)
    assert oracle.zone_layout(2**32 - 1, 32, 8) == (32, 24)
    # bits at or above hi are ignored (they are shared by the whole subproblem)
    assert oracle.zone_layout(0xFF000005, 24, 2) == (3, 1)
    assert oracle.zone_layout(2**64 - 1, 64, 10) == (64, 54)


def test_bucket_order_is_zone_order():
    rs = np.random.RandomState(8)
    keys = rs.randint(0, 2**32, size=20_000, dtype=np.uint64).astype(W32)
    heavy = np.unique(keys[:40]).astype(np.uint64)
    ids, nb = oracle.bucket_ids(heavy, int(keys.max()), 32, 5, keys)
    zone = keys >> 27
    # buckets never mix zones and follow zone order
    for z in range(32):
        zi = ids[zone == z]
        zo = ids[zone != z]
        if len(zi):
            assert not np.isin(zi, zo).any()
    o = np.argsort(ids, kind="stable")
    assert np.all(np.diff(zone[o].astype(np.int64)) >= 0)
    # every heavy key has its own bucket
    for h in heavy:
        sel = ids[keys == h]
        assert len(np.unique(sel)) == 1
        assert np.sum(ids == sel[0]) == np.sum(keys == h)


# ----------------------------------------------------------------- DTMerge
def _zone(rs, n0, m, heavy_max):
    # heavy keys never occur among the light keys (GetBucketId sends every
    # record of a heavy key to its heavy bucket): light keys even, heavy odd
    light = (np.sort(rs.randint(0, 1000, size=n0)) * 2).astype(np.uint64)
    hk = np.sort(rs.choice(np.arange(1, 2001, 2), size=m,
                           replace=False)).astype(np.uint64)
    hs = rs.randint(1, heavy_max + 1, size=m).astype(np.int64)
    return light, hk, hs


@pytest.mark.parametrize("heavy_scale", [3, 400])
def test_dtmerge_equals_stable_sort(heavy_scale):
    rs = np.random.RandomState(heavy_scale)
    for trial in range(60):
        n0 = rs.randint(0, 300)
        m = rs.randint(1, 12)
        light, hk, hs = _zone(rs, n0, m, heavy_scale)
        nh = int(hs.sum())
        lv = np.arange(n0, dtype=np.uint64)
        hv = np.arange(n0, n0 + nh, dtype=np.uint64)
        keys, vals, copied = oracle.dtmerge(light, lv, hk, hs, hv)
        allk = np.concatenate([light, np.repeat(hk, hs)]).astype(np.uint64)
        allv = np.concatenate([lv, hv])
        ek, ev = oracle.stable_sort(allk, allv)
        np.testing.assert_array_equal(keys, ek)
        np.testing.assert_array_equal(vals, ev)
        # DTMerge copies only the smaller side out of place
        assert copied == min(n0, nh)
        assert copied <= (n0 + nh) // 2


# ------------------------------------------------------- planted mistakes
ORACLE_SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    # ties broken by descending original index -> unstable
    "reversed_ties": ("  return a->idx < b->idx;\n}",
                      "  return a->idx > b->idx;\n}"),
    # signed 32-bit compare
    "signed_keys": ("if (a->key != b->key) return a->key < b->key;",
                    "if (a->key != b->key) return (int32_t)a->key < (int32_t)b->key;"),
    # values not gathered by the sorted order
    "ungathered_values": ("((const uint32_t *)vcopy)[x[i].idx]",
                          "((const uint32_t *)vcopy)[i]"),
    # last merge round drops the odd run
    "lost_run": ("if (runs % 2) bound[nr++] = bound[runs - 1];",
                 "if (runs % 2 && 0) bound[nr++] = bound[runs - 1];"),
    # subsample positions shifted to 0, L, 2L, ...
    "subsample_offset": ("uint64_t a = s[(j + 1) * L - 1], b = s[(j + 2) * L - 1];",
                         "uint64_t a = s[j * L], b = s[(j + 1) * L];"),
    # heavy buckets numbered before the light bucket of their zone
    "heavy_first": ("if (a->light != b->light) return a->light > b->light;",
                    "if (a->light != b->light) return a->light < b->light;"),
    # overflow test off by one bit
    "overflow_bit": ("} else if (((key & mhi) >> t) != 0 && t < 64) {",
                     "} else if (((key & mhi) >> (t + 1)) != 0 && t < 63) {"),
    # DTMerge rotation with a single flip
    "one_flip": ("        rec_flip(A, s, s + sz);\n        rec_flip(A, d, s + sz);",
                 "        rec_flip(A, d, s + sz);"),
    # stable position counts ties after j as well
    "position_ties": ("c += (ki < kj) || (ki == kj && i < j);",
                      "c += (ki < kj) || (ki == kj && i <= j);"),
    # key-only check: a run may take more input keys than it is long
    "run_overuse": ("if (lo == r || rk[lo] != k || rlen[lo] == 0) ok = 0;",
                    "if (lo == r || rk[lo] != k) ok = 0;"),
    # key-only check: the run search finds the first run above the key
    "run_upper_bound": ("if (rk[mid] < k) lo = mid + 1; else hi = mid;",
                        "if (rk[mid] <= k) lo = mid + 1; else hi = mid;"),
}


def _run_pins():
    """The pins above, as one function that raises on the first failure."""
    test_brute_force_all_small_inputs(W32)
    test_brute_force_length6_sampled()
    test_invariants_u32_families("uniform")
    test_invariants_u32_families("distinct10")
    test_extreme_keys()
    test_stable_positions_match_definition()
    test_heavy_rule_hand_example()
    test_bucket_ids_hand_example_r16_gamma2()
    test_golden_overflow_bucket_example()
    test_dtmerge_equals_stable_sort(3)
    test_dtmerge_equals_stable_sort(400)
    test_check_sorted_keys_brute_force(W32)


def test_pins_pass_on_the_oracle():
    _run_pins()


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistakes_are_caught(mutant, tmp_path):
    src = open(ORACLE_SRC).read()
    old, new = MUTANTS[mutant]
    assert src.count(old) == 1, "mutation anchor not found: " + mutant
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                           "-pthread", str(mpath), "-o", str(so)])
    with oracle.using_library(str(so)):
        with pytest.raises(AssertionError):
            _run_pins()


def test_golden_example_catches_the_overflow_mistake(tmp_path):
    # the paper's overflow example alone fails on the oracle built with its
    # overflow test off by one bit
    src = open(ORACLE_SRC).read()
    old, new = MUTANTS["overflow_bit"]
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                           "-pthread", str(mpath), "-o", str(so)])
    with oracle.using_library(str(so)):
        with pytest.raises(AssertionError):
            test_golden_overflow_bucket_example()


# ------------------------------------------------ check of a claimed output
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_check_stable_accepts_exactly_the_stable_sort(dtype):
    # the checker (the definition read as a test) against numpy's stable
    # argsort, and against plausible wrong outputs, each caught
    n = 200_003
    keys = gen.family("zipf1.2hash" if dtype == np.uint64 else "zipf1.0", n, dtype, seed=17)
    order = np.argsort(keys, kind="stable")
    ko, io = keys[order], order.astype(np.uint64 if dtype == np.uint64 else np.uint32)
    assert oracle.check_stable(keys, ko, io) == -1
    # two records of equal key in the wrong order
    i = int(np.where(ko[1:] == ko[:-1])[0][0])
    bad = io.copy()
    bad[i], bad[i + 1] = bad[i + 1], bad[i]
    assert oracle.check_stable(keys, ko, bad) == i
    # two records of different keys swapped (keys and indices together)
    j = int(np.where(ko[1:] != ko[:-1])[0][0])
    kb, ib = ko.copy(), io.copy()
    kb[j], kb[j + 1] = kb[j + 1], kb[j]
    ib[j], ib[j + 1] = ib[j + 1], ib[j]
    assert oracle.check_stable(keys, kb, ib) == j
    # one record duplicated over its neighbour
    dup = io.copy()
    dup[j + 1] = dup[j]
    assert oracle.check_stable(keys, ko, dup) >= 0
    # a key changed, or an index out of range
    kx = ko.copy()
    kx[n // 2] ^= dtype(1)
    assert oracle.check_stable(keys, kx, io) >= 0
    ix = io.copy()
    ix[-1] = n
    assert oracle.check_stable(keys, ko, ix) == n - 1


@pytest.mark.parametrize("dtype", [W32, W64])
def test_check_sorted_keys_brute_force(dtype):
    # every candidate output of every tiny input, over keys from four
    # different top-16-bit groups: exactly the sorted input passes
    top = int(np.iinfo(dtype).max)
    half = 1 << (8 * np.dtype(dtype).itemsize - 1)
    alphabet = [0, 1, half, top]
    for n in range(0, 4):
        for combo in itertools.product(alphabet, repeat=n):
            keys = np.array(combo, dtype=dtype)
            want = sorted(combo)
            for cand in itertools.product(alphabet, repeat=n):
                got = oracle.check_sorted_keys(keys, np.array(cand, dtype=dtype), nthreads=1)
                assert (got == -1) == (list(cand) == want), (combo, cand, got)


@pytest.mark.parametrize("dtype", [W32, W64])
def test_check_sorted_keys_catches_wrong_outputs(dtype):
    # the key-only checker against numpy's sort and plausible wrong outputs
    n = 200_003
    keys = gen.family("zipf1.2hash" if dtype == W64 else "zipf1.0", n, dtype, seed=19)
    ko = np.sort(keys)
    assert oracle.check_sorted_keys(keys, ko) == -1
    assert oracle.check_sorted_keys(keys, ko, nthreads=3) == -1
    # the input itself (unsorted)
    assert oracle.check_sorted_keys(keys, keys) >= 0
    # two neighbours of different keys swapped
    j = int(np.where(ko[1:] != ko[:-1])[0][0])
    kb = ko.copy()
    kb[j], kb[j + 1] = kb[j + 1], kb[j]
    assert oracle.check_sorted_keys(keys, kb) == j
    # a run one longer and the next one shorter, order kept (same group)
    kr = ko.copy()
    kr[j + 1] = kr[j]
    if (int(ko[j]) >> 16) == (int(ko[j + 1]) >> 16) or dtype == W64:
        assert oracle.check_sorted_keys(keys, kr) >= 0
    # one key replaced by a neighbouring value that the input lacks
    ks = ko.copy()
    absent = int(ko[-1]) - 1
    while absent in set(ko[-50:].tolist()):
        absent -= 1
    ks[-1] = absent
    ks.sort()
    assert oracle.check_sorted_keys(keys, ks) >= 0
    # the largest key moved to another top-16-bit group, order kept
    kg = ko.copy()
    kg[-1] = np.iinfo(dtype).max if int(ko[-1]) != np.iinfo(dtype).max else 0
    kg.sort()
    assert oracle.check_sorted_keys(keys, kg) >= 0
    # every key one larger
    assert oracle.check_sorted_keys(keys, ko + dtype(1)) >= 0


def test_edge_list_generator():
    # the graph-transpose workload: sources non-decreasing with about E/V
    # out-edges each, destinations Zipf(1) over V vertices (the busiest one
    # takes about 1/H_V of the edges), and the stable sort by destination
    # keeps each destination's sources increasing
    n = 1_000_000
    V = gen.EDGE_VERTICES
    dst = gen.family("edges", n, np.uint32, seed=1)
    src = gen.edge_src(n, np.uint32)
    assert int(dst.max()) < V
    assert (np.diff(src.astype(np.int64)) >= 0).all()
    assert src[0] == 0 and int(src[-1]) == (n - 1) * V // n
    _, cnt = np.unique(dst, return_counts=True)
    H = np.log(V) + 0.5772156649
    assert abs(cnt.max() / n - 1.0 / H) < 0.1 / H
    k, v = oracle.stable_sort(dst, src)
    same = k[1:] == k[:-1]
    assert (v[1:][same] >= v[:-1][same]).all()

