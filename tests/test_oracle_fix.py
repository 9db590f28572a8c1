"""Pins for the oracle's full correction loop (Sec. 4): hand-worked golden
cases, special cases with known answers, invariants on random fields,
termination under adversarial inputs, and a brute-force check of the
troublemaker set (Sec. 4.2)."""
import glob
import json
import os

import numpy as np
import pytest

import oracle
from paper_2406_09423_gb300 import synth
from tests import bruteforce as bf
from tests.invariants import bits_of, check_result, within_bound

GOLDEN = sorted(p for p in glob.glob(os.path.join(os.path.dirname(__file__), "golden", "*.json"))
                if not os.path.basename(p).startswith("fullsize_"))  # hand-worked cases only


@pytest.mark.parametrize("path", GOLDEN, ids=[os.path.basename(p) for p in GOLDEN])
def test_golden_hand_worked(path):
    case = json.load(open(path))
    dt = np.dtype(case["dtype"])
    shape = tuple(case["shape"])
    f = np.array(case["f"], dtype=dt).reshape(shape)
    fhat = np.array(case["fhat"], dtype=dt).reshape(shape)
    r = oracle.fix(f, fhat, case["xi"], trace_cap=1000)
    assert r.status == 0
    assert np.array_equal(r.g.reshape(-1), np.array(case["g"], dtype=dt))
    assert list(r.edit_idx) == case["edit_idx"]
    for k, v in case["counts"].items():
        assert r.counts[k] == v, k
    assert r.trace.tolist() == case["trace"]
    check_result(f, fhat, case["xi"], r.g, r.edit_idx, r.edit_val, r.label_max, r.label_min)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("shape", [(16, 16), (5, 6, 7)])
def test_identity_input_needs_no_edits(dtype, shape):
    f = np.random.default_rng(1).standard_normal(shape).astype(dtype)
    r = oracle.fix(f, f.copy(), 0.1)
    assert r.status == 0 and len(r.edit_idx) == 0
    c = r.counts
    assert c["sweeps"] == 1 and c["c_passes"] == 1 and c["label_evals"] == 1
    assert c["r_rounds"] == 0 and c["dec_edits"] == 0 and c["freezes"] == 0


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_exact_shift_preserves_order(dtype):
    # values on a 1/1024 grid shifted by exactly 2^-9: every comparison is
    # unchanged, so the segmentation already agrees and nothing is edited.
    rng = np.random.default_rng(2)
    f = (rng.integers(-2000, 2000, (12, 13)) / 1024.0).astype(dtype)
    fhat = (f - dtype(2.0 ** -9)).astype(dtype)
    r = oracle.fix(f, fhat, 2.0 ** -8)
    assert r.status == 0 and len(r.edit_idx) == 0 and r.counts["sweeps"] == 1


def test_zero_bound_forces_identity():
    f = np.random.default_rng(3).standard_normal((6, 6)).astype(np.float32)
    assert oracle.fix(f, f.copy(), 0.0).status == 0
    bad = f.copy()
    bad[2, 3] = np.nextafter(bad[2, 3], np.float32(10))
    assert oracle.fix(f, bad, 0.0).status == -4


def test_input_validation():
    f = np.zeros((4, 4), dtype=np.float32)
    g = f.copy()
    g[1, 1] = np.nan
    assert oracle.fix(f, g, 0.1).status == -3
    assert oracle.fix(g, f, 0.1).status == -3
    g = f.copy()
    g[0, 0] = 0.2
    assert oracle.fix(f, g, 0.1).status == -4
    assert oracle.fix(f, f, -1.0).status == -1
    assert oracle.fix(f, f, float("nan")).status == -1


def _random_case(rng, shape, dtype, rel):
    kind = rng.integers(0, 3)
    if kind == 0:
        f = rng.standard_normal(shape)
    elif kind == 1:  # smooth
        f = np.cumsum(np.cumsum(rng.standard_normal(shape), axis=-1), axis=0)
    else:  # plateaus in f itself
        f = rng.integers(0, 5, shape).astype(np.float64)
    f = f.astype(dtype)
    xi = synth.xi_for(f, rel)
    return f, synth.quantise(f, xi), xi


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("shape", [(7, 9), (16, 12), (1, 17), (4, 5, 6), (6, 6, 6), (3, 1, 8)])
@pytest.mark.parametrize("rel", [1e-3, 1e-2, 1e-1])
def test_random_fields_satisfy_invariants(dtype, shape, rel):
    rng = np.random.default_rng(abs(hash((shape, rel, str(dtype)))) % 2 ** 32)
    for _ in range(3):
        f, fhat, xi = _random_case(rng, shape, dtype, rel)
        r = oracle.fix(f, fhat, xi)
        assert r.status == 0
        check_result(f, fhat, xi, r.g, r.edit_idx, r.edit_val, r.label_max, r.label_min)
        assert r.counts["edits"] == len(r.edit_idx)
        assert r.counts["label_evals"] == r.counts["r_rounds"] + 1


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("shape", [(10, 10), (5, 5, 5)])
def test_constant_decompression_terminates(dtype, shape):
    # A bound as large as the range admits a constant decompressed field:
    # every vertex but one is wrong. The loop must still end with a valid result.
    rng = np.random.default_rng(4)
    f = rng.uniform(0, 1, shape).astype(dtype)
    fhat = np.full(shape, 0.5, dtype=dtype)
    r = oracle.fix(f, fhat, 1.0)
    assert r.status == 0
    check_result(f, fhat, 1.0, r.g, r.edit_idx, r.edit_val)


def test_lower_bound_collision_forces_freezes():
    # f values one ulp apart with a huge bound: their lower bounds round to the
    # same float, so decreasing edits alone cannot restore the order; the
    # freeze guard must fire and the result must still be correct.
    one = np.float32(1.0)
    vals = [one]
    for _ in range(15):
        vals.append(np.nextafter(vals[-1], np.float32(2)))
    f = np.array(vals[::-1], dtype=np.float32).reshape(4, 4)  # decreasing with index
    xi = float(np.float32(2.0 ** 20))
    fhat = np.full((4, 4), 1.0, dtype=np.float32)  # equal values: index order wins
    r = oracle.fix(f, fhat, xi)
    assert r.status == 0
    assert r.counts["freezes"] > 0
    check_result(f, fhat, xi, r.g, r.edit_idx, r.edit_val)


def _rounds_case(name):
    if name == "bumps":
        f = synth.bumps2d(24, 20, 3)
        xi = synth.xi_for(f, 1e-2)
        return f, synth.quantise(f, xi), xi
    if name == "turb3d":
        f = synth.turbulence3d(12, 2, kmax=3.0, shape=(9, 10, 12))
        xi = synth.xi_for(f, 3e-2)
        return f, synth.quantise(f, xi), xi
    rng = np.random.default_rng(5)  # constant decompression: freezes
    f = rng.uniform(0, 1, (7, 8)).astype(np.float32)
    return f, np.full(f.shape, 0.5, dtype=np.float32), 1.0


@pytest.mark.parametrize("name", ["bumps", "turb3d", "constant"])
def test_every_round_lowers_or_freezes(name):
    # The convergence argument with the freeze guard (Sec. 4.3): after every
    # round g stays within the bound (Eq. 1), each vertex's value only
    # decreases or is reset to f once and then never changes, and a round
    # changes every vertex it decreases plus at most the ones it freezes.
    # g after k rounds is the result of a run capped at k rounds.
    f, fhat, xi = _rounds_case(name)
    full = oracle.fix(f, fhat, xi, max_rounds=5000, trace_cap=100000)  # these cases need < 100
    assert full.status == 0
    trace = full.trace
    assert len(trace) > 1
    prev = fhat.reshape(-1)
    reset = np.zeros(prev.size, dtype=bool)
    fb = bits_of(f)
    for k in range(1, len(trace) + 1):
        gk = oracle.fix(f, fhat, xi, max_rounds=k - 1).g.reshape(-1)
        assert within_bound(f.reshape(-1), gk, xi)
        changed = bits_of(gk) != bits_of(prev)
        up = gk > prev
        assert not (changed & reset).any(), "a reset vertex changed again"
        assert ((gk < prev) | (bits_of(gk) == fb))[changed].all(), "a value rose above its previous one"
        assert (bits_of(gk) == fb)[up].all(), "a rise that is not a reset to f"
        _, _, _, nd, nf = trace[k - 1]
        assert nd <= changed.sum() <= nd + nf
        reset |= up
        prev = gk
    assert np.array_equal(bits_of(prev), bits_of(full.g))


def test_fig5_event_chain():
    # Sec. 4.2, Fig. 5: f_i > f_j > f_k with g_j > g_i > g_k at first. The
    # FNmax at i is fixed by lowering j; i then descends through j in g but
    # through k in f, a troublemaker fixed by lowering k; k becomes an FPmin,
    # fixed (Eq. 3, the neighbour maximal in g) by lowering i, which brings
    # back an FNmax at i. Rebuilt on a 5x3 grid (x fastest, xi = 8, so
    # lb = f - 8): i = 7 at the centre, j = 6 to its left, k = 8 to its
    # right; f has maxima {0, 7} and minima {5, 9}. Every value worked by hand.
    f = np.array([[12, 9, 8, 6, 3], [1, 7, 10, 4, 0], [2, 5, 9, 6, 2]], dtype=np.float64)
    fhat = f.copy()
    fhat.flat[[6, 7, 8, 9, 12]] = [9.5, 9, 5, 1, 8]
    xi, i, j, k = 8.0, 7, 6, 8
    assert f.flat[i] > f.flat[j] > f.flat[k] and fhat.flat[j] > fhat.flat[i] > fhat.flat[k]
    up_f, dn_f = oracle.directions(f)
    assert dn_f[i] == k
    g = [fhat.reshape(-1)] + [oracle.fix(f, fhat, xi, max_rounds=q).g.reshape(-1) for q in range(3)]

    def edits(q):
        return {int(v): float(g[q + 1][v]) for v in np.flatnonzero(g[q + 1] != g[q])}

    # round 1 (C): the FNmax at i is the only false case; j: 9.5 -> (9.5 + -1) / 2
    b0 = oracle.false_bits(f, fhat)
    assert {int(v): int(b0[v]) for v in np.flatnonzero(b0)} == {i: 4}
    assert edits(0) == {j: 4.25}
    # round 2 (R): no false case; i is the only troublemaker, a descending
    # one (g: 7 -> 6 -> 5, f: 7 -> 8 -> 9); k: 5 -> (5 + -4) / 2
    assert not oracle.false_bits(f, g[1].reshape(f.shape)).any()
    t1 = oracle.troublemakers(f, g[1].reshape(f.shape))
    assert {int(v): int(t1[v]) for v in np.flatnonzero(t1)} == {i: 2}
    assert edits(1) == {k: 0.5}
    # round 3 (C): k is an FPmin (and its neighbour 9 an FNmin); the FPmin
    # sub-loop lowers i, k's highest neighbour: 9 -> (9 + 2) / 2
    b2 = oracle.false_bits(f, g[2].reshape(f.shape))
    assert {int(v): int(b2[v]) for v in np.flatnonzero(b2)} == {k: 2, 9: 8}
    assert edits(2) == {i: 5.5}
    # then i is an FNmax again (its neighbour 1 holds 9)
    assert oracle.false_bits(f, g[3].reshape(f.shape))[i] & 4
    full = oracle.fix(f, fhat, xi, max_rounds=5000, trace_cap=1000)
    assert full.status == 0
    assert [tuple(int(x) for x in t[:3]) for t in full.trace[:3]] == [(0, 2, 1), (1, 0, 1), (0, 1, 1)]
    check_result(f, fhat, xi, full.g, full.edit_idx, full.edit_val, full.label_max, full.label_min)


def test_troublemakers_are_first_discrepancies():
    # With equal extremum sets, the troublemaker set must equal the set of
    # first vertices, along each wrongly labelled vertex's integral line in f,
    # where the steepest neighbour in g differs from that in f (Sec. 4.2).
    rng = np.random.default_rng(8)
    tested = 0
    for trial in range(4000):
        shape = [(4, 4), (5, 6), (3, 3, 3), (2, 4, 3)][trial % 4]
        f = rng.standard_normal(shape)
        g = f + rng.normal(0, 0.35, shape)
        adj = bf.adjacency(shape)
        fu, fd = bf.directions(f, adj)
        gu, gd = bf.directions(g, adj)
        if bf.extrema(fu, fd) != bf.extrema(gu, gd):
            continue
        M, Mg = bf.walk_labels(fu), bf.walk_labels(gu)
        m, mg = bf.walk_labels(fd), bf.walk_labels(gd)
        want_a, want_d = set(), set()
        for v in range(f.size):
            if M[v] != Mg[v]:
                w = v
                while gu[w] == fu[w]:
                    assert fu[w] != w
                    w = fu[w]
                want_a.add(w)
            if m[v] != mg[v]:
                w = v
                while gd[w] == fd[w]:
                    assert fd[w] != w
                    w = fd[w]
                want_d.add(w)
        if not want_a and not want_d:
            continue
        bits = oracle.troublemakers(f, g)
        assert set(np.flatnonzero(bits & 1)) == want_a
        assert set(np.flatnonzero(bits & 2)) == want_d
        tested += 1
        if tested >= 60:
            break
    assert tested >= 20


def test_bumps128_workload_invariants():
    f = synth.bumps2d()
    xi = synth.xi_for(f, 1e-3)
    fhat = synth.quantise(f, xi)
    r = oracle.fix(f, fhat, xi)
    assert r.status == 0
    check_result(f, fhat, xi, r.g, r.edit_idx, r.edit_val, r.label_max, r.label_min)
