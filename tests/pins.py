"""Pins of the oracle against facts that do not come from the oracle itself.

Each check returns normally when it holds and raises AssertionError when it
does not. They are collected by ``test_oracle_pins.py`` and re-run against
deliberately broken copies of the oracle by ``test_oracle_mutants.py``, which
shows that a plausible slip in the oracle trips at least one of them.

The independent references used here:
  * brute force with a different formula: Pearson correlation from
    ``numpy.corrcoef`` and d = sqrt(2 m (1 - rho)), with the argmin taken by a
    stable sort (equivalent to the z-normalised Euclidean distance for
    non-constant windows, population std);
  * closed forms (affine images, sine vs cosine over a full period, constant
    windows);
  * invariants (range [0, 2 sqrt(m)], affine invariance, planted copies, the
    segment-boundary rule of Def. 8, the per-segment decomposition of
    Algorithm 2);
  * the paper's guarantees for a dictionary cut from T_B: Lemma 1
    (P_hat >= P) and Lemma 2 (P_hat - P <= e_max, e_max by its definition in
    Sec. 3.3);
  * what the paper's illustration of Algorithm 2 (Sec. 3.2) shows: repeated
    patterns found exactly, the unique pattern as the profile's maximum.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
import synthetic

TOL = 1e-9


def _valid_windows(offsets, m):
    gs = []
    for s in range(len(offsets) - 1):
        for o in range(0, int(offsets[s + 1] - offsets[s]) - m + 1):
            gs.append(int(offsets[s]) + o)
    return np.array(gs, dtype=np.int64)


def brute_force(query, dict_samples, offsets, m):
    """Independent all-pairs join via numpy.corrcoef (non-constant windows only)."""
    q = np.asarray(query, dtype=np.float64)
    b = np.asarray(dict_samples, dtype=np.float64)
    gs = _valid_windows(offsets, m)
    nq = len(q) - m + 1
    D = np.empty((nq, len(gs)))
    for r in range(nq):
        for c, g in enumerate(gs):
            rho = np.corrcoef(q[r : r + m], b[g : g + m])[0, 1]
            D[r, c] = math.sqrt(max(0.0, 2 * m * (1 - rho)))
    order = np.argsort(D, axis=1, kind="stable")  # stable: lowest g among equals
    best = D[np.arange(nq), order[:, 0]]
    second = D[np.arange(nq), order[:, 1]] if len(gs) > 1 else np.full(nq, np.inf)
    return best, gs[order[:, 0]], second


def pin_brute_force(lib, seeds=range(6)):
    for seed in seeds:
        rng = np.random.default_rng(1000 + seed)
        m = int(rng.choice([3, 4, 8]))
        na = int(rng.integers(m, 48))
        nseg = int(rng.integers(1, 4))
        lens = rng.integers(max(1, m - 2), 20, nseg)
        offs = np.concatenate(([0], np.cumsum(lens))).astype(np.int64)
        q = rng.standard_normal(na)
        b = rng.standard_normal(int(offs[-1]))
        d, i, d2 = oracle.ab_join(q, b, offs, m, lib=lib)
        if len(_valid_windows(offs, m)) == 0:
            assert np.all(np.isinf(d)) and np.all(i == -1)
            continue
        bd, bi, bd2 = brute_force(q, b, offs, m)
        np.testing.assert_allclose(d, bd, rtol=0, atol=1e-9)
        np.testing.assert_allclose(d2, bd2, rtol=0, atol=1e-9)
        uniq = (bd2 - bd) > 1e-9
        assert np.array_equal(i[uniq], bi[uniq])


def pin_closed_forms(lib):
    m = 32
    t = np.arange(m)
    x = np.sin(2 * np.pi * t / m) + 0.3 * np.cos(6 * np.pi * t / m) + 0.01 * t
    # affine image with positive scale: the same z-normalised shape
    assert oracle.pair_distance(x, 3.5 * x - 7.0, lib=lib) < 1e-6
    # negative scale: z(y) = -z(x), so d = |2 z(x)| = 2 sqrt(m)
    assert abs(oracle.pair_distance(x, -0.5 * x + 1.0, lib=lib) - 2 * math.sqrt(m)) < 1e-9
    # sine and cosine over one full period are orthogonal: rho = 0, d = sqrt(2m)
    s = np.sin(2 * np.pi * t / m)
    c = np.cos(2 * np.pi * t / m)
    assert abs(oracle.pair_distance(s, c, lib=lib) - math.sqrt(2 * m)) < 1e-9
    # constant windows: zero z-vector
    k = np.full(m, 4.25)
    assert abs(oracle.pair_distance(k, x, lib=lib) - math.sqrt(m)) < 1e-12
    assert abs(oracle.pair_distance(x, k, lib=lib) - math.sqrt(m)) < 1e-12
    assert oracle.pair_distance(k, np.full(m, -1.0), lib=lib) == 0.0
    # a window of equal values whose float mean is not exactly that value is
    # still constant
    assert oracle.pair_distance(np.full(m, 0.1), np.full(m, 0.7), lib=lib) == 0.0
    # m = 2: two non-constant windows are either the same (+) or opposite (-) shape
    assert oracle.pair_distance([0.0, 1.0], [5.0, 9.0], lib=lib) < 1e-12
    assert abs(oracle.pair_distance([0.0, 1.0], [9.0, 5.0], lib=lib) - 2 * math.sqrt(2)) < 1e-12
    # a hand-computed value: x = [0, 0, 3], y = [0, 3, 0]; z(x) = [-1, -1, 2]/sqrt(2),
    # z(y) = [-1, 2, -1]/sqrt(2); difference [0, -3, 3]/sqrt(2); squared norm 9
    assert abs(oracle.pair_distance([0.0, 0.0, 3.0], [0.0, 3.0, 0.0], lib=lib) - 3.0) < 1e-12


def pin_stats(lib):
    rng = np.random.default_rng(7)
    x = rng.standard_normal(200) * 3 + 100
    m = 17
    mu, sd, cst = oracle.window_stats(x, m, lib=lib)
    from numpy.lib.stride_tricks import sliding_window_view

    W = sliding_window_view(x, m)
    np.testing.assert_allclose(mu, W.mean(axis=1), rtol=1e-13)
    np.testing.assert_allclose(sd, W.std(axis=1, ddof=0), rtol=1e-10)
    assert not cst.any()
    y = np.concatenate([np.full(20, 2.0), rng.standard_normal(10)])
    _, _, cst = oracle.window_stats(y, 8, lib=lib)
    assert cst[:13].all() and not cst[13:].any()


def pin_invariants(lib):
    w = synthetic.workload("rw_fp64_4k", scale=0.125)
    q, b, offs, m = w.query, w.dict_samples, w.offsets, 32
    d, i, d2 = oracle.ab_join(q, b, offs, m, lib=lib)
    # range
    assert np.all(d >= 0) and np.all(d <= 2 * math.sqrt(m) + 1e-12)
    uniq = (d2 - d) > 1e-7
    # affine invariance of the query
    da, ia, _ = oracle.ab_join(2.5 * q + 40.0, b, offs, m, lib=lib)
    np.testing.assert_allclose(da, d, atol=1e-7)
    assert np.array_equal(ia[uniq], i[uniq])
    # per-segment affine maps of the dictionary
    b2 = b.copy()
    for s in range(len(offs) - 1):
        b2[offs[s] : offs[s + 1]] = (0.5 + s) * b2[offs[s] : offs[s + 1]] - 3.0 * s
    db, ib, _ = oracle.ab_join(q, b2, offs, m, lib=lib)
    np.testing.assert_allclose(db, d, atol=1e-7)
    assert np.array_equal(ib[uniq], i[uniq])
    # Algorithm 2: per-segment joins merged by an element-wise minimum
    best = np.full(len(d), np.inf)
    arg = np.full(len(d), -1, dtype=np.int64)
    for s in range(len(offs) - 1):
        seg = b[offs[s] : offs[s + 1]]
        if len(seg) < m:
            continue
        ds, is_, _ = oracle.ab_join(q, seg, np.array([0, len(seg)]), m, lib=lib)
        better = ds < best
        best = np.where(better, ds, best)
        arg = np.where(better, is_ + offs[s], arg)
    np.testing.assert_array_equal(best, d)
    np.testing.assert_array_equal(arg, i)


def pin_planted_and_boundary(lib):
    rng = np.random.default_rng(11)
    m = 24
    b = rng.standard_normal(3 * 100).cumsum()
    offs = np.array([0, 100, 200, 300], dtype=np.int64)
    q = rng.standard_normal(400).cumsum()
    # exact copy of dictionary window (segment 1, offset 37) planted at row 150
    g = int(offs[1]) + 37
    q[150 : 150 + m] = b[g : g + m]
    # a window straddling the junction between segments 1 and 2 planted at row 300
    j = int(offs[2]) - m // 2
    q[300 : 300 + m] = b[j : j + m]
    d, i, d2 = oracle.ab_join(q, b, offs, m, lib=lib)
    assert d[150] <= 1e-6 and i[150] == g
    # the straddling window is not a dictionary window (Def. 8), so it is not found...
    assert d[300] > 0.05 and i[300] != j
    # ...but it is found once the two segments are one element
    d1, i1, _ = oracle.ab_join(q, b, np.array([0, 100, 300], dtype=np.int64), m, lib=lib)
    assert d1[300] <= 1e-6 and i1[300] == j
    # a single segment equal to T_B is the exact AB join; index is a window of T_B
    dx, ix, _ = oracle.ab_join(q, b, np.array([0, len(b)]), m, lib=lib)
    assert np.all(dx <= d + 1e-12)


def pin_lemmas(lib):
    """Lemma 1 and Lemma 2 for a dictionary cut from T_B (Proposition 1 holds)."""
    for name, m in (("ecg", 64), ("rw", 32)):
        if name == "ecg":
            tb = synthetic.ecg_like(6000, 21)
            ta = synthetic.ecg_like(1500, 22, n_malformed=3)
        else:
            tb = synthetic.random_walk(6000, 23)
            ta = synthetic.random_walk(1500, 24)
        db, offs = synthetic.cut_dictionary(tb, 12, 200)
        P, _, _ = oracle.ab_join(ta, tb, np.array([0, len(tb)]), m, lib=lib)
        Ph, _, _ = oracle.ab_join(ta, db, offs, m, lib=lib)
        # e_max = max over windows of T_B of NNDist(window, D_{B,m})
        e, _, _ = oracle.ab_join(tb, db, offs, m, lib=lib)
        e_max = e.max()
        assert np.all(Ph >= P - 1e-9), "Lemma 1 (no false negatives) violated"
        assert np.all(Ph - P <= e_max + 1e-9), "Lemma 2 (max error) violated"
        assert e_max > 0 and (Ph - P).max() > 0  # the dictionary really is lossy here


def pin_empty(lib):
    q = np.arange(10.0)
    d, i, d2 = oracle.ab_join(q, np.arange(9.0), np.array([0, 3, 6, 9]), 4, lib=lib)
    assert np.all(np.isinf(d)) and np.all(i == -1) and np.all(np.isinf(d2))
    # one window only: the second-best is +inf
    d, i, d2 = oracle.ab_join(q, np.arange(9.0) ** 2, np.array([0, 4]), 4, lib=lib)
    assert np.all(i == 0) and np.all(np.isinf(d2))


def pin_constant_rows(lib):
    m = 8
    b = np.concatenate([np.arange(20.0) ** 1.5, np.full(12, 3.0), np.sin(np.arange(20.0))])
    offs = np.array([0, 20, 32, 52], dtype=np.int64)
    q = np.concatenate([np.full(10, -2.0), np.cos(np.arange(30.0))])
    d, i, _ = oracle.ab_join(q, b, offs, m, lib=lib)
    # row 0..2 are constant query windows: nearest is the first constant dictionary window
    assert np.all(d[:3] == 0.0) and np.all(i[:3] == 20)
    # without constant dictionary windows, a constant query window is sqrt(m) from everything,
    # and the lowest index wins the tie
    d, i, _ = oracle.ab_join(q, b[:20], np.array([0, 20]), m, lib=lib)
    assert np.allclose(d[:3], math.sqrt(m), atol=1e-12) and np.all(i[:3] == 0)


def pin_correlation_output(lib, seeds=range(4)):
    """The correlation form against numpy.corrcoef maxima, and the constant-window reading."""
    for seed in seeds:
        rng = np.random.default_rng(2000 + seed)
        m = int(rng.choice([4, 6, 8]))
        na = int(rng.integers(m + 4, 40))
        lens = rng.integers(m, 18, int(rng.integers(1, 4)))
        offs = np.concatenate(([0], np.cumsum(lens))).astype(np.int64)
        q = rng.standard_normal(na)
        b = rng.standard_normal(int(offs[-1]))
        rho, i = oracle.ab_join_corr(q, b, offs, m, lib=lib)
        gs = _valid_windows(offs, m)
        R = np.array([[np.corrcoef(q[r : r + m], b[g : g + m])[0, 1] for g in gs] for r in range(na - m + 1)])
        np.testing.assert_allclose(rho, R.max(axis=1), rtol=0, atol=1e-9)
        top2 = np.sort(R, axis=1)[:, -2:] if len(gs) > 1 else None
        uniq = (top2[:, 1] - top2[:, 0]) > 1e-9 if top2 is not None else np.ones(len(rho), bool)
        assert np.array_equal(i[uniq], gs[np.argmax(R, axis=1)][uniq])
    # constant windows: 0.5 against non-constant windows, 1 against a constant one
    m = 6
    b = np.concatenate([np.sin(np.arange(30.0)), np.full(10, 2.0)])
    q = np.concatenate([np.full(8, -1.0), np.cos(np.arange(20.0))])
    rho, i = oracle.ab_join_corr(q, b[:30], np.array([0, 30]), m, lib=lib)
    assert np.allclose(rho[:3], 0.5, atol=1e-12) and np.all(i[:3] == 0)
    rho, i = oracle.ab_join_corr(q, b, np.array([0, 30, 40]), m, lib=lib)
    assert np.all(rho[:3] == 1.0) and np.all(i[:3] == 30)
    # no window at all: -inf / -1
    rho, i = oracle.ab_join_corr(q, np.arange(9.0), np.array([0, 3, 6, 9]), m, lib=lib)
    assert np.all(np.isneginf(rho)) and np.all(i == -1)


def _bf_dist_matrix(x, m):
    """All-pairs z-normalised distances of one series' windows via numpy.corrcoef (non-constant windows)."""
    nq = len(x) - m + 1
    W = np.array([x[i : i + m] for i in range(nq)])
    R = np.corrcoef(W)
    return np.sqrt(np.maximum(0.0, 2 * m * (1 - R)))


def pin_self_join(lib, seeds=range(4)):
    for seed in seeds:
        rng = np.random.default_rng(3000 + seed)
        m = int(rng.choice([4, 6, 8]))
        x = rng.standard_normal(int(rng.integers(3 * m, 50))).cumsum()
        D = _bf_dist_matrix(x, m)
        nq = len(D)
        for excl in (1, (m + 1) // 2, m):
            d, i = oracle.self_join(x, m, excl, lib=lib)
            g = np.arange(nq)
            Dm = np.where(np.abs(g[None, :] - g[:, None]) < excl, np.inf, D)
            bd = Dm.min(axis=1)
            np.testing.assert_allclose(d, bd, rtol=0, atol=1e-9)
            srt = np.sort(Dm, axis=1)
            uniq = np.isfinite(bd) & ((srt[:, 1] - srt[:, 0]) > 1e-9)
            assert np.array_equal(i[uniq], np.argmin(Dm, axis=1)[uniq])
            assert np.all(i[~np.isfinite(bd)] == -1)


def _bf_learn(x, m, k, budget):
    """Algorithm 1 restated on brute-force distances (memory terminal condition)."""
    D = _bf_dist_matrix(x, m)
    nq = len(D)
    g = np.arange(nq)
    P = np.where(np.abs(g[None, :] - g[:, None]) < (m + 1) // 2, np.inf, D).min(axis=1)
    S = np.zeros(nq)
    taken = np.zeros(nq, bool)
    pad = int(np.floor((k - 1) * m / 2))
    chosen, cover = [], np.zeros(len(x), bool)
    while True:
        Pp = np.where(taken, np.inf, P - S)
        if not np.isfinite(Pp).any():
            break
        j = int(np.argmin(Pp))
        chosen.append(j)
        cover[max(0, j - pad) : min(len(x), j + m + pad)] = True
        taken[max(0, j - m // 2) : min(nq, j + m // 2)] = True
        S = D[j] if len(chosen) == 1 else np.minimum(S, D[j])
        if cover.sum() >= budget:
            break
    return chosen


def pin_learn_dictionary(lib):
    rng = np.random.default_rng(4000)
    # against an independent restatement on brute-force distances
    for m, n, budget in ((8, 120, 60), (6, 90, 40)):
        x = rng.standard_normal(n).cumsum()
        segs, chosen, smax = oracle.learn_dictionary(x, m, 1.5, "memory", budget, lib=lib)
        assert chosen == _bf_learn(x, m, 1.5, budget)
    # invariants on a longer series with a planted motif
    m = 16
    x = rng.standard_normal(600).cumsum()
    motif = np.sin(np.linspace(0, 3 * np.pi, m)) * 5
    x[100:116] = motif + x[99]
    x[420:436] = motif * 2 + x[419]
    P, _ = oracle.self_join(x, m, (m + 1) // 2, lib=lib)
    segs, chosen, smax = oracle.learn_dictionary(x, m, 1.5, "memory", 150, lib=lib)
    assert chosen[0] == int(np.argmin(P)) and chosen[0] in (100, 420)
    for a in range(len(chosen)):
        for b in range(a):
            assert not (chosen[b] - m // 2 <= chosen[a] < chosen[b] + m // 2)
    total = sum(L for _, L in segs)
    assert total >= 150
    pad = int(np.floor(0.5 * m / 2))
    before = oracle._merge([(max(0, j - pad), min(len(x), j + m + pad)) for j in chosen[:-1]])
    assert sum(b - a for a, b in before) < 150
    starts = [a for a, _ in segs]
    assert starts == sorted(starts) and all(a + L <= b for (a, L), (b, _) in zip(segs, segs[1:]))
    # the learned dictionary's e_max stays within the reported bound max(S)
    samples = np.concatenate([x[a : a + L] for a, L in segs])
    offs = np.concatenate(([0], np.cumsum([L for _, L in segs])))
    d, _, _ = oracle.ab_join(x, samples, offs, m, lib=lib)
    assert d.max() <= smax + 1e-9
    # the e_max terminal condition, with a target the memory-limited run reached: the greedy
    # picks are the same, so the e_max run stops no later and with max(S) <= target
    segs_m, chosen_m, target = oracle.learn_dictionary(x, m, 1.5, "memory", 400, lib=lib)
    segs, chosen, smax = oracle.learn_dictionary(x, m, 1.5, "emax", target, lib=lib)
    assert smax <= target and len(chosen) <= len(chosen_m) and chosen == chosen_m[: len(chosen)]
    d, _, _ = oracle.ab_join(x, np.concatenate([x[a : a + L] for a, L in segs]),
                             np.concatenate(([0], np.cumsum([L for _, L in segs]))), m, lib=lib)
    assert d.max() <= target + 1e-9


def pin_dictionary_figure(lib):
    """The illustration of Algorithm 2 (Sec. 3.2, the figure of the dictionary join).

    T_A repeats three patterns and holds one unique pattern; the dictionary has
    one element per repeated pattern. Expected from the method: every window
    lying inside an occurrence of a repeated pattern is found exactly (distance
    0, at the same offset of the element holding that pattern); P_hat is the
    element-wise minimum of the per-element profiles P_AD[i]; and P_hat's
    largest value falls on a window that overlaps the unique pattern. The
    repeated patterns are smooth (random-walk bridges) and the unique one is
    white noise, so its windows correlate with no dictionary window.
    """
    rng = np.random.default_rng(31)
    L, m = 96, 16
    ramp = np.linspace(0.0, 1.0, L)
    pats = []
    for _ in range(3):
        w = rng.standard_normal(L).cumsum()
        pats.append(w - w[0] - ramp * (w[-1] - w[0]))  # starts and ends at 0
    unique = rng.standard_normal(L)
    order = [0, 1, 2, 1, 0, 2, None, 2, 0, 1]
    q = np.concatenate([unique if k is None else pats[k] for k in order])
    b = np.concatenate(pats)
    offs = np.array([0, L, 2 * L, 3 * L], dtype=np.int64)
    d, i, _ = oracle.ab_join(q, b, offs, m, lib=lib)
    for n, k in enumerate(order):
        if k is None:
            continue
        for o in range(L - m + 1):
            r = n * L + o
            assert d[r] == 0.0 and i[r] == offs[k] + o, (n, k, o, d[r], i[r])
    per = [oracle.ab_join(q, pats[k], np.array([0, L]), m, lib=lib)[0] for k in range(3)]
    assert np.array_equal(np.minimum(np.minimum(per[0], per[1]), per[2]), d)
    a0 = order.index(None) * L
    top = int(np.argmax(d))
    assert a0 - m + 1 <= top <= a0 + L - 1, (top, a0)


ALL_PINS = (
    pin_brute_force,
    pin_closed_forms,
    pin_stats,
    pin_invariants,
    pin_planted_and_boundary,
    pin_lemmas,
    pin_empty,
    pin_constant_rows,
    pin_correlation_output,
    pin_self_join,
    pin_learn_dictionary,
    pin_dictionary_figure,
)
