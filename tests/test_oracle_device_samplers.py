"""Pins of the oracle's device-precision pair samplers, the checkers the GPU's indices are
compared with bit for bit (CPU only):

  * Algorithm 8 on FP32 ratios (uniform proposals, accept iff u < r);
  * Algorithm 7 on FP32 ratios (B steps from (n, n), move iff fl32(u r(I, J)) < r(I*, J*));
  * the rejection sampler with factorised proposals (rows and columns drawn by their own
    weights, accept iff u < acc);
  * the systematic variant of the three-stage sampler, and the FP64 systematic sampler.

Each is checked against the exact finite law its definition fixes (tests/exact_laws.py,
numpy only) by chi-square, and against tie cases built from the Philox words of a slot's
first attempt (the oracle's Philox is pinned to the published known-answer vectors).  A
planted mistake -- compiled into a copy of the oracle, never into the oracle itself -- must
fail these pins: a non-strict comparison, the uniform taken from the wrong Philox word, the
attempt counter off by one, a Metropolis-Hastings chain started at (0, 0), a systematic
offset that is not random, and a column stage that reuses the tile stage's word.
"""
import numpy as np
import pytest
from scipy import stats

from exact_laws import U23_STEPS, accept_count, chi2_pvalue, kp_law, kp_mh_transition, q24
from oracle import core

SEED = 0x1234_5678_9ABC
RS, MH, SYS, RSF, RSU = 3, 4, 5, 6, 7


def words(slot, gid, purpose, j, seed=SEED, base=0):
    """Philox4x32-10 words of the counter (slot, gid, purpose | base << 4, j)."""
    return core.philox([slot, gid, purpose | (base << 4), j], [seed & 0xFFFFFFFF, seed >> 32])


def u23(w):
    return np.float32(((int(w) >> 9) + 0.5) * 2.0 ** -23)


def idx(w, N):
    return (int(w) * N) >> 32


@pytest.fixture(scope="module")
def mutants(tmp_path_factory):
    """Copies of the oracle, each with one planted mistake."""
    plants = {
        "rs_le": [("if (u < ratio[(size_t)I * N + J]) { ok = 1; ++a; break; }",
                   "if (u <= ratio[(size_t)I * N + J]) { ok = 1; ++a; break; }")],
        "rs_lane": [("      float u = (float)u23(w[2]);\n      if (u < ratio",
                     "      float u = (float)u23(w[3]);\n      if (u < ratio")],
        "rs_attempt": [("draw(seed_lo, seed_hi, (uint32_t)n, gid, ORC_PURPOSE_RS, base, a, w);",
                        "draw(seed_lo, seed_hi, (uint32_t)n, gid, ORC_PURPOSE_RS, base, a + 1, w);")],
        "mh_origin": [("    int I = n % N, J = n % N;\n    float cur = ratio",
                       "    int I = 0, J = 0;\n    float cur = ratio")],
        "mh_le": [("      if (lhs < prop) {", "      if (lhs <= prop) {")],
        "rsf_le": [("if (u < acc[(size_t)I * N + J]) { ok = 1; ++a; break; }",
                    "if (u <= acc[(size_t)I * N + J]) { ok = 1; ++a; break; }")],
        "sys_fixed": [("int64_t f = inverse_cdf(C, E, NN, ((double)n + U) / (double)N);",
                       "int64_t f = inverse_cdf(C, E, NN, ((double)n + 0.5) / (double)N);")],
        "kpsys_word": [("    int kt = fixed_pick_rem(q, nT, w2, &w3);",
                        "    int kt = fixed_pick_rem(q, nT, w2, &w3);\n    w3 = w2;")],
    }
    out = {}
    for name, rep in plants.items():
        d = tmp_path_factory.mktemp(name)
        out[name] = core.load_variant(core.build_variant(rep, str(d)))
    return out


# ------------------------------------------------------------ Algorithm 8, FP32 ratios
def rs_ratio_case(N=4, seed=3):
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.0, 1.0, (N, N)).astype(np.float32)
    r[1, 2] = 0.0                       # never accepted
    r[3, 0] = np.float32(2.0 ** -20)    # a rare pair
    r[0, 1] = 1.0                       # always accepted when proposed
    return r


def check_rs_law(lib_ctx, slots=200_000):
    r = rs_ratio_case()
    with lib_ctx:
        li, ri, att, st = core.kp_rs_pairs(r, SEED, 9, 0, slots)
    assert st == 0
    a = accept_count(r)
    P = a / a.sum()
    p_law = chi2_pvalue(li, ri, P)
    # attempts per slot are geometric with success N^-2 sum_ij a_ij / 2^23
    p_acc = a.sum() / U23_STEPS / r.size
    z = (att.mean() - 1 / p_acc) / (np.sqrt(1 - p_acc) / p_acc / np.sqrt(slots))
    return p_law, abs(z)


class _Same:
    def __enter__(self):
        return None

    def __exit__(self, *e):
        return False


def rs_tie_mismatches(lib_ctx, N=5, gid=17, slots=24):
    """Slot n's first proposal (I0, J0) gets the ratio u0 of its own first attempt: the strict
    test rejects it (at least two attempts); one ulp above u0 accepts it at once."""
    bad = 0
    for n in range(slots):
        w = words(n, gid, RS, 0)
        I0, J0, u0 = idx(w[0], N), idx(w[1], N), u23(w[2])
        for ratio0, expect_first in ((u0, False), (np.nextafter(u0, np.float32(1)), True)):
            r = np.ones((N, N), np.float32)
            r[I0, J0] = ratio0
            with lib_ctx:
                li, ri, att, st = core.kp_rs_pairs(r, SEED, gid, n, n + 1)
            first = att[0] == 1 and li[0] == I0 and ri[0] == J0
            bad += int(first != expect_first)
    return bad


def test_kp_rs_exact_law_and_attempts():
    p, z = check_rs_law(_Same())
    assert p > 1e-3 and z < 5, (p, z)


def test_kp_rs_strict_comparison_and_philox_words():
    assert rs_tie_mismatches(_Same()) == 0


def test_kp_rs_cap_leaves_no_index():
    r = np.full((4, 4), np.float32(2.0 ** -30))
    li, ri, att, st = core.kp_rs_pairs(r, SEED, 1, 0, 8, max_attempts=32)
    assert st == 8 and (att == 32).all() and (li == -1).all() and (ri == -1).all()


@pytest.mark.parametrize("name", ["rs_le", "rs_lane", "rs_attempt"])
def test_kp_rs_pins_reject_planted_mistakes(mutants, name):
    assert rs_tie_mismatches(core.variant(mutants[name])) > 0


# ------------------------------------------------------------ Algorithm 7, FP32 ratios
def mh_draws(lib_ctx, r, n_start, B, G, gid=5):
    N = r.shape[0]
    with lib_ctx:
        li, ri = core.kp_mh_pairs(r, SEED, gid, 0, N * G, B)
    sel = np.arange(N * G) % N == n_start
    return li[sel], ri[sel]


def mh_ratio_case():
    return np.array([[0.25, 0.5, 0.0], [0.75, 0.125, 0.25], [0.0, 0.25, 0.5]], np.float32)


def mh_law_pvalues(lib_ctx, G=40_000):
    r = mh_ratio_case()
    P = kp_mh_transition(r)
    out = []
    for n_start, B in ((1, 1), (2, 2), (1, 3)):
        s0 = n_start * 3 + n_start
        law = np.linalg.matrix_power(P, B)[s0].reshape(3, 3)
        li, ri = mh_draws(lib_ctx, r, n_start, B, G)
        out.append(chi2_pvalue(li, ri, law))
    return out


def mh_tie_mismatches(lib_ctx, N=4, gid=23, slots=24):
    """Slot n's first proposal (n != n mod N pair) weighs exactly fl32(u0 r_start): the strict
    rule stays at (n, n) after one step; one ulp more moves."""
    bad = checked = 0
    for n in range(slots):
        w = words(n, gid, MH, 0)
        Is, Js, u0 = idx(w[0], N), idx(w[1], N), u23(w[2])
        s = n % N
        if (Is, Js) == (s, s):
            continue
        checked += 1
        cur = np.float32(0.5)
        tie = np.float32(u0 * cur)
        for prop, moves in ((tie, False), (np.nextafter(tie, np.float32(1)), True)):
            r = np.full((N, N), np.float32(0.5))
            r[Is, Js] = prop
            with lib_ctx:
                li, ri = core.kp_mh_pairs(r, SEED, gid, n, n + 1, 1)
            moved = (li[0], ri[0]) == (Is, Js)
            stayed = (li[0], ri[0]) == (s, s)
            bad += int(not (moved if moves else stayed))
    assert checked >= 10
    return bad


def test_kp_mh_chain_law():
    ps = mh_law_pvalues(_Same())
    assert min(ps) > 1e-3, ps


def test_kp_mh_strict_move_rule():
    assert mh_tie_mismatches(_Same()) == 0


def test_kp_mh_pins_reject_planted_mistakes(mutants):
    assert min(mh_law_pvalues(core.variant(mutants["mh_origin"]), G=20_000)) < 1e-6
    assert mh_tie_mismatches(core.variant(mutants["mh_le"])) > 0


# ------------------------------------------------------------ factorised proposals
def rsf_case(N=5, seed=8):
    rng = np.random.default_rng(seed)
    ra = rng.uniform(0.05, 1.0, N).astype(np.float32)
    ra[ra.argmax()] = 1.0
    ra[2] = 0.0                                   # a row never proposed
    rc = rng.uniform(0.0, 1.0, N).astype(np.float32) ** 3
    rc[rc.argmax()] = 1.0
    acc = rng.uniform(0.0, 1.0, (N, N)).astype(np.float32)
    acc[0, 3] = 0.0
    return ra, rc, acc


def test_kp_rsf_exact_law_and_attempts():
    ra, rc, acc = rsf_case()
    slots = 200_000
    li, ri, att, st = core.kp_rsf_pairs(ra, rc, acc, SEED, 4, 0, slots)
    assert st == 0
    Rq = np.floor(ra.astype(np.float64) * 2.0 ** 40)
    Cq = np.floor(rc.astype(np.float64) * 2.0 ** 40)
    g = np.outer(Rq / Rq.sum(), Cq / Cq.sum())
    a = accept_count(acc) / U23_STEPS
    assert chi2_pvalue(li, ri, g * a) > 1e-3
    p_acc = (g * a).sum()
    z = (att.mean() - 1 / p_acc) / (np.sqrt(1 - p_acc) / p_acc / np.sqrt(slots))
    assert abs(z) < 5, z


def rsf_tie_mismatches(lib_ctx, N=5, gid=31, slots=24):
    ra = np.ones(N, np.float32)
    rc = np.ones(N, np.float32)
    bad = 0
    for n in range(slots):
        w = words(n, gid, RSF, 0)
        v = words(n, gid, RSU, 0)
        # uniform proposal images: I = floor(U1 S / 2^64) / 2^40 with S = N 2^40
        U1 = (int(w[0]) << 32) | int(w[1])
        U2 = (int(w[2]) << 32) | int(w[3])
        I0 = ((U1 * (N << 40)) >> 64) >> 40
        J0 = ((U2 * (N << 40)) >> 64) >> 40
        u0 = u23(v[0])
        for a0, expect_first in ((u0, False), (np.nextafter(u0, np.float32(1)), True)):
            acc = np.ones((N, N), np.float32)
            acc[I0, J0] = a0
            with lib_ctx:
                li, ri, att, st = core.kp_rsf_pairs(ra, rc, acc, SEED, gid, n, n + 1)
            first = att[0] == 1 and li[0] == I0 and ri[0] == J0
            bad += int(first != expect_first)
    return bad


def test_kp_rsf_strict_comparison_and_philox_words():
    assert rsf_tie_mismatches(_Same()) == 0


def test_kp_rsf_pins_reject_planted_mistake(mutants):
    assert rsf_tie_mismatches(core.variant(mutants["rsf_le"])) > 0


def test_fp64_factorised_rejection_law():
    """FP64: target exp(la_i + lc_j + lacc_ij) with lacc <= 0; expected attempts
    sum_i e^la_i sum_j e^lc_j / sum_ij e^(la_i + lc_j + lacc_ij)."""
    rng = np.random.default_rng(12)
    N = 4
    la = rng.normal(0, 1, N)
    lc = rng.normal(0, 2, N)
    lacc = -rng.exponential(1.5, (N, N))
    lacc[2, 1] = -np.inf
    slots = 150_000
    li, ri, att, st = core.rsf_pairs(la, lc, lacc, SEED, 2, 0, slots)
    assert st == 0
    Wt = np.exp(la[:, None] + lc[None, :] + lacc)
    assert chi2_pvalue(li, ri, Wt / Wt.sum()) > 1e-3
    expect = np.exp(la).sum() * np.exp(lc).sum() / Wt.sum()
    assert att / slots == pytest.approx(expect, rel=0.03)


# ------------------------------------------------------------ systematic resampling
def sys_matrix(N=4, seed=21):
    rng = np.random.default_rng(seed)
    logW = rng.normal(0, 1.2, (N, N))
    logW[1, 3] = -np.inf
    return logW


def sys_stats(lib_ctx, logW, G=4000):
    """Per combination (gid): pair counts of the N slots.  Systematic positions (k + U) / N
    put every count at floor or ceil of N P_ij; over many U the mean count is N P_ij."""
    N = logW.shape[0]
    P = np.exp(logW - logW.max())
    P /= P.sum()
    counts = np.zeros((G, N * N))
    with lib_ctx:
        for g in range(G):
            li, ri = core.sys_pairs(logW, SEED, g, 0, N)
            counts[g] = np.bincount(li * N + ri, minlength=N * N)
    target = N * P.ravel()
    within = np.all(np.abs(counts - target) < 1 + 1e-9)
    z = np.abs(counts.mean(0) - target) / (0.5 / np.sqrt(G))
    return within, z.max()


def test_systematic_counts_and_mean():
    within, zmax = sys_stats(_Same(), sys_matrix())
    assert within and zmax < 5, zmax


def test_systematic_pins_reject_planted_mistake(mutants):
    within, zmax = sys_stats(core.variant(mutants["sys_fixed"]), sys_matrix())
    assert zmax > 20


def kp_sys_case(N=7, B=3, seed=5):
    rng = np.random.default_rng(seed)
    nT = (N + B - 1) // B
    r = rng.uniform(0.05, 1, N).astype(np.float32)
    r[4] = 0.0
    r[r.argmax()] = 1.0
    e = rng.uniform(0, 1, (N, N)).astype(np.float32)
    e[:, 5] = 0.0
    t = np.stack([[e[i, k * B:(k + 1) * B].sum() for k in range(nT)] for i in range(N)]).astype(np.float32)
    return r, t, e, B


def kp_sys_stats(lib_ctx, G=6000):
    r, t, e, B = kp_sys_case()
    N = r.shape[0]
    P = kp_law(r, t, e, B)
    target = N * P.ravel()
    counts = np.zeros((G, N * N))
    with lib_ctx:
        for g in range(G):
            li, ri = core.kp_sys_pairs(r, t, e, B, SEED, g, 0, N)
            counts[g] = np.bincount(li * N + ri, minlength=N * N)
    within = np.all(np.abs(counts - target) < 1 + 1e-6)
    z = np.abs(counts.mean(0) - target) / (0.5 / np.sqrt(G))
    return within, z.max(), counts


def test_kp_systematic_counts_and_mean():
    within, zmax, counts = kp_sys_stats(_Same())
    assert within and zmax < 5, zmax
    assert counts[:, 4 * 7:5 * 7].sum() == 0 and counts.reshape(-1, 7, 7)[:, :, 5].sum() == 0


def test_kp_systematic_pins_reject_planted_mistake(mutants):
    within, zmax, _ = kp_sys_stats(core.variant(mutants["kpsys_word"]))
    assert (not within) or zmax > 10, zmax


def test_kp_systematic_images_match_q24():
    """The tile and column images used are the q24 images of the three-stage sampler: with
    all row weight on one row and one tile, slot positions step through the column images."""
    N = B = 8
    e = np.zeros((N, N), np.float32)
    e[2] = np.array([1, 2, 3, 4, 0, 6, 7, 1], np.float32) * np.float32(1e-3)
    t = e.sum(1, keepdims=True).astype(np.float32)
    r = np.zeros(N, np.float32)
    r[2] = 1.0
    q = q24(e[2], t[2, 0])
    for g in range(50):
        li, ri = core.kp_sys_pairs(r, t, e, B, SEED, g, 0, N)
        assert (li == 2).all()
        c = np.bincount(ri, minlength=N)
        assert np.all(np.abs(c - N * q / q.sum()) < 1 + 1e-6)
