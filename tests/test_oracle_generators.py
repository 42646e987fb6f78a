"""Pins of the CPU oracle's generators against facts fixed by the paper and by
mathematics (no GPU).  Each test names the passage it pins."""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# --------------------------------------------------------------- seeding
def test_splitmix64_known_answer():
    """SplitMix64 (Steele, Lea & Flood 2014), the seeding reading of Sec. III.B:
    the generator's published output for state 1234567 advanced by the golden
    gamma before each output."""
    got = [oracle.splitmix64(1234567, i) for i in range(5)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_taus_seeds_valid_and_distinct():
    """Taus seeds must leave every Tausworthe word out of its absorbing set
    (y1 >= 2, y2 >= 8, y3 >= 16: the masked bits of Algorithm 1 need one set)."""
    g = oracle.Gen("taus", 1234, 100000)
    st = g.state
    assert (st[:, 0] >= 2).all() and (st[:, 1] >= 8).all() and (st[:, 2] >= 16).all()
    assert len(np.unique(st.view(np.uint64).reshape(-1, 2), axis=0)) == 100000


# ------------------------------------------------------------- Hybrid Taus
def _bits_word(bits, start):
    w = 0
    for j in range(32):
        w = (w << 1) | bits[start + j]
    return w


@pytest.mark.parametrize("which,k,q,s", [(0, 31, 13, 12), (1, 29, 2, 4), (2, 28, 3, 17)])
def test_taus_component_matches_bit_recurrence(which, k, q, s):
    """Eq. 2 defines the Tausworthe bits by a linear recurrence mod 2; with the
    trinomial z^k - z^q - 1 it reads b_n = b_{n-(k-q)} xor b_{n-k}, and word n
    holds bits b_{ns} .. b_{ns+31} (most significant first).  The fast word
    word step of Algorithm 1 must reproduce it for every n >= 1."""
    rng = np.random.default_rng(7 + which)
    for _ in range(4):
        a0 = int(rng.integers(0, 2**32))
        bits = [(a0 >> (31 - i)) & 1 for i in range(k)]
        while len(bits) < 60 * s + 40:
            n = len(bits)
            bits.append(bits[n - (k - q)] ^ bits[n - k])
        a = a0
        for n in range(1, 60):
            a = oracle.taus_component(a, which)
            assert a == _bits_word(bits, n * s), (which, n)


@pytest.mark.parametrize("which,period", [(0, 2**31 - 1), (1, 2**29 - 1), (2, 2**28 - 1)])
def test_taus_component_periods(which, period):
    """Sec. II.C: the Tausworthe periods are 2^k - 1 for k = 31, 29, 28 (the
    printed p2 = 2^30 - 1 disagrees with the 29-bit mask 4294967288 of
    Appendix A; brute force settles it).  Counted by iterating the word step."""
    assert oracle.taus_component_period(which, 0xDEADBEEF) == period


def test_taus_lcg_full_period_and_first_values():
    """Appendix A: LCG a=1664525, c=1013904223 mod 2^32 (Eq. 1).  Hull-Dobell
    gives the full period 2^32; the first values from 0 follow from Eq. 1."""
    a, c = 1664525, 1013904223
    assert c % 2 == 1 and (a - 1) % 4 == 0
    assert oracle.lcg_period(12345) == 2**32
    y = np.zeros(4, np.uint32)
    oracle.taus_next(y)
    assert int(y[3]) == 0x3C6EF35F
    oracle.taus_next(y)
    assert int(y[3]) == (a * 0x3C6EF35F + c) % 2**32 == 0x47502932


def test_taus_combined_period_claim():
    """Sec. II.C claims a combined period ~2^121 > 10^36; with the brute-forced
    component periods (pairwise coprime) the product is ~2^120 > 10^36."""
    p = [2**31 - 1, 2**29 - 1, 2**28 - 1, 2**32]
    for i in range(4):
        for j in range(i + 1, 4):
            assert math.gcd(p[i], p[j]) == 1
    assert math.prod(p) > 10**36


def test_taus_output_advances_before_output():
    """Algorithm 1: words are advanced first, then the output is
    their xor.  From the all-zero Tausworthe words the output is the LCG word."""
    y = np.array([0, 0, 0, 5], np.uint32)
    out = oracle.taus_next(y)
    assert out == (1664525 * 5 + 1013904223) % 2**32


# -------------------------------------------------------------------- Ran2
M1, A1, M2, A2 = 2147483563, 40014, 2147483399, 40692


def test_ran2_schrage_equals_modular_product():
    """Algorithm 2 computes a*x mod m by Schrage's factorisation."""
    rng = np.random.default_rng(3)
    for which, (m, a) in enumerate([(M1, A1), (M2, A2)]):
        xs = list(rng.integers(1, m, 2000)) + [1, 2, m - 1, m - 2, m // a, m // a + 1]
        for x in xs:
            assert oracle.ran2_schrage(int(x), which) == (a * int(x)) % m


def _factor(n):
    f, d = [], 2
    while d * d <= n:
        while n % d == 0:
            f.append(d)
            n //= d
        d += 1
    if n > 1:
        f.append(n)
    return sorted(set(f))


def test_ran2_components_full_period():
    """Each L'Ecuyer component must have period m-1 (a primitive root mod the
    prime m); with lcm(m1-1, m2-1) > 2e18 this is the period of Sec. II.B."""
    for m, a in [(M1, A1), (M2, A2)]:
        assert all(m % d for d in range(2, math.isqrt(m) + 1))      # m prime
        assert pow(a, m - 1, m) == 1
        for q in _factor(m - 1):
            assert pow(a, (m - 1) // q, m) != 1
    assert math.lcm(M1 - 1, M2 - 1) > 2 * 10**18


def test_ran2_output_range_and_shuffle_conservation():
    """Algorithm 2: every output iy lies in [1, m1-1]; the shuffle table stores
    each idum once and hands it back once (iy = iv[j] - idum2, wrapped by
    m1-1), so  {initial iv} + {idum_1..n} = {retrieved values} + {final iv}
    as multisets.  idum/idum2 are recomputed independently as plain
    multiplicative LCG sequences."""
    g = oracle.Gen("ran2", 99, 3)
    for s in range(3):
        st = g.state[s].copy()
        iv0 = st[3:].tolist()
        idum, idum2 = int(st[0]), int(st[1])
        retrieved, produced = [], []
        for _ in range(20000):
            idum = (A1 * idum) % M1
            idum2 = (A2 * idum2) % M2
            iy = oracle.ran2_next(st)
            assert 1 <= iy <= M1 - 1
            assert int(st[0]) == idum and int(st[1]) == idum2
            w = iy + idum2
            retrieved.append(w if w <= M1 - 1 else w - (M1 - 1))
            produced.append(idum)
        assert sorted(iv0 + produced) == sorted(retrieved + st[3:].tolist())


NDIV = 1 + (M1 - 1) // 32


def _band_repeat_violations(outputs, idums, idum2s):
    """A consequence of the Bays-Durham shuffle (Knuth, TAOCP vol. 2, Sec.
    3.2.2, Algorithm B; the draw of Algorithm 2) that needs no table state:
    the slot a draw reads and refills is the one the previous output selects,
    so when outputs y_{n-1} and y_n fall in the same band floor(y / NDIV),
    draw n+1 reads back the idum that draw n stored there:
        y_{n+1} = idum_n - idum2_{n+1}   (wrapped into [1, m1-1]).
    Returns (band repeats seen, repeats where that fails)."""
    seen = bad = 0
    for n in range(1, len(outputs) - 1):
        if outputs[n - 1] // NDIV != outputs[n] // NDIV:
            continue
        seen += 1
        want = idums[n] - idum2s[n + 1]
        if want < 1:
            want += M1 - 1
        bad += outputs[n + 1] != want
    return seen, bad


def _lcg_sequence(x, a, m, n):
    out = []
    for _ in range(n):
        x = (a * x) % m
        out.append(x)
    return out


def test_ran2_shuffle_slot_chosen_by_previous_output():
    """Algorithm 2's draw takes the table slot from the previous output iy
    (j = iy / NDIV before iy is replaced).  Pinned from outside the oracle's
    formula: its outputs, with idum and idum2 recomputed here as plain
    multiplicative LCG sequences, satisfy the band-repeat property above at
    every repeat, while CPU models of the same draw that take the slot from
    the new idum, the new idum2 or the old idum fail it at most repeats."""
    draws = 20000
    g = oracle.Gen("ran2", 4242, 2)
    for s in range(2):
        st = g.state[s].copy()
        init = st.copy()
        outs = [int(st[2])] + [int(oracle.ran2_next(st)) for _ in range(draws)]
        idums = [int(init[0])] + _lcg_sequence(int(init[0]), A1, M1, draws)
        idum2s = [int(init[1])] + _lcg_sequence(int(init[1]), A2, M2, draws)
        seen, bad = _band_repeat_violations(outs, idums, idum2s)
        assert seen > draws // 64 and bad == 0, (seen, bad)

    # planted mistakes (CPU models, not the oracle): the slot from another word
    def mutant(pick):
        st = [int(v) for v in init]
        iv = st[3:]
        idum, idum2, iy = st[0], st[1], st[2]
        outs = [iy]
        for _ in range(draws):
            old_idum = idum
            idum = (A1 * idum) % M1
            idum2 = (A2 * idum2) % M2
            j = {"idum": idum, "idum2": idum2, "old_idum": old_idum}[pick] // NDIV
            iy = iv[j] - idum2
            iv[j] = idum
            if iy < 1:
                iy += M1 - 1
            outs.append(iy)
        return outs

    for pick in ("idum", "idum2", "old_idum"):
        seen, bad = _band_repeat_violations(mutant(pick), idums, idum2s)
        assert seen > draws // 64 and bad > seen // 2, (pick, seen, bad)


def test_ran2_init_warmup():
    """Algorithm 2's seeding: idum2 = seed, NTAB+8 Schrage steps, the last NTAB
    stored with iv[j] at j = NTAB-1 .. 0; iy starts as iv[0] (reading)."""
    g = oracle.Gen("ran2", 5, 2)
    for s in range(2):
        w = oracle.splitmix64(5, 8 * s)
        seed = 1 + w % (M1 - 1)
        st = g.state[s]
        assert int(st[1]) == seed
        x, seq = seed, []
        for _ in range(40):
            x = (A1 * x) % M1
            seq.append(x)
        # j = 39 .. 0; iv[j] for j < 32 gets the value of step 40-j (1-based)
        assert [int(v) for v in st[3:]] == [seq[39 - j] for j in range(32)]
        assert int(st[0]) == seq[-1] and int(st[2]) == int(st[3])


# ------------------------------------------------------- Lagged Fibonacci
def _golden_rows():
    rows = []
    with open(os.path.join(GOLDEN, "table1_lags.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(map(int, line.split())))
    return rows


def test_lfg_table_matches_paper():
    """Table I as printed, except row 4 whose printed sl = 12470 gives a
    reducible trinomial; it is read as 13470 (next test)."""
    for r, sl, ll in _golden_rows():
        assert oracle.lfg_table(r) == ((13470, ll) if r == 4 else (sl, ll))


def test_lfg_table_row4_printed_value_reducible():
    """x^23209 + x^12470 + 1 (Table I row 4 as printed) is reducible, so it
    cannot give the maximal period Sec. II.D requires; 13470 (one digit away)
    and its reciprocal exponent 9739 give irreducible trinomials."""
    assert not oracle.gf2_trinomial_irreducible(23209, 12470)
    assert oracle.gf2_trinomial_irreducible(23209, 13470)
    assert oracle.gf2_trinomial_irreducible(23209, 9739)


def _lucas_lehmer(p):
    m = (1 << p) - 1
    s = 4
    for _ in range(p - 2):
        s = (s * s - 2) % m
    return s == 0


@pytest.mark.parametrize("row", [0, 1, 2, 3, 4, 5, 6])
def test_lfg_table_rows_primitive(row):
    """Sec. II.D: ll a Mersenne exponent and x^ll + x^sl + 1 primitive.  For
    prime ll, irreducible + 2^ll - 1 prime => primitive.  Checked live for the
    smaller rows (Lucas-Lehmer for ll <= 23209)."""
    sl, ll = oracle.lfg_table(row)
    assert oracle.gf2_trinomial_irreducible(ll, sl)
    if ll <= 23209:
        assert _lucas_lehmer(ll)


def test_lfg_table_large_rows_primitive_stored():
    """Rows 7-9 (ll up to 3021377) take minutes each; their irreducibility was
    computed by tests/golden/make_goldens.py with the same oracle routine."""
    path = os.path.join(GOLDEN, "table1_irreducible.txt")
    if not os.path.exists(path):
        pytest.skip("golden not generated")
    rows = {}
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                r, sl, ll, ok = map(int, line.split())
                rows[r] = (sl, ll, ok)
    for r in (7, 8, 9):
        sl, ll = oracle.lfg_table(r)
        assert rows[r] == (sl, ll, 1)


def test_gf2_irreducibility_small_brute_force():
    """The GF(2) routine agrees with trial division for all small trinomials."""
    def pmod(a, b):
        db = b.bit_length() - 1
        while a and a.bit_length() - 1 >= db:
            a ^= b << (a.bit_length() - 1 - db)
        return a

    def irred(p):
        d = p.bit_length() - 1
        return all(pmod(p, q) for q in range(2, 1 << (d // 2 + 1)) if q.bit_length() - 1 <= d // 2)

    for ll in [3, 5, 7, 11, 13]:
        for k in range(1, ll):
            assert oracle.gf2_trinomial_irreducible(ll, k) == irred((1 << ll) | (1 << k) | 1)


def _lsb_period(sl, ll, seed):
    g = oracle.Gen.custom_lfg(seed, sl, ll)
    n = 4 * (2**ll)
    bits = g.fill_u32(n) & 1
    tail = bits[-ll:]
    for p in range(1, 2**ll + 1):
        if np.array_equal(bits[n - ll - p:n - p], tail):
            return p
    return None


@pytest.mark.parametrize("sl,ll,primitive", [(3, 7, True), (4, 7, True), (1, 7, True),
                                             (2, 7, False), (2, 5, True)])
def test_lfg_lsb_period_tiny_lags(sl, ll, primitive):
    """Algorithm 3 mod 2^32: the least significant bits follow the GF(2)
    recurrence of the trinomial, so their period is 2^ll - 1 exactly when the
    trinomial is primitive (Sec. II.D)."""
    p = _lsb_period(sl, ll, 11)
    if primitive:
        assert p == 2**ll - 1
    else:
        assert p != 2**ll - 1


def test_lfg_ring_matches_linear_history():
    """Algorithm 3 on a ring of ll words (slot p mod ll) equals the plain
    linear recurrence x_p = x_{p-ll} + x_{p-(ll-sl)} mod 2^32 kept as a full
    history array (brute force on tiny and on Table I lags)."""
    for sl, ll in [(4, 7), (3, 7), (1252, 2281)]:
        g = oracle.Gen.custom_lfg(5, sl, ll)
        hist = [int(v) for v in g.state]          # hist[q + ll] = x_q
        n = 5 * ll + 13
        got = g.fill_u32(n)
        for p in range(n):
            hist.append((hist[p] + hist[p + sl]) % 2**32)
        assert [int(v) for v in got] == hist[ll:]
        assert np.array_equal(g.ring_in_order(), np.array(hist[-ll:], np.uint32))


def test_lfg_ring_matches_linear_history_random_lags_and_splits():
    """The same identity for 40 random lag pairs (sl < ll up to 300) and fills
    split at random lengths (including zero and lengths beyond several ll):
    the ring position carried across calls never loses or repeats a value."""
    rng = np.random.default_rng(77)
    for _ in range(40):
        ll = int(rng.integers(2, 300))
        sl = int(rng.integers(1, ll))
        g = oracle.Gen.custom_lfg(int(rng.integers(0, 2**31)), sl, ll)
        hist = [int(v) for v in g.state]
        got = []
        for _ in range(int(rng.integers(1, 6))):
            got += [int(v) for v in g.fill_u32(int(rng.integers(0, 4 * ll)))]
        for p in range(len(got)):
            hist.append((hist[p] + hist[p + sl]) % 2**32)
        assert got == hist[ll:]
        assert np.array_equal(g.ring_in_order(), np.array(hist[-ll:], np.uint32))


def test_lfg_default_row_selection():
    """Table I picks a row by system size; with 4 numbers per thread per step
    the row needs sl > 4N and ll - sl > 4N, else the last row (reading)."""
    assert oracle.lfg_default_row(1) == 0
    assert oracle.lfg_default_row(256) == 0        # 1024 < 1029
    assert oracle.lfg_default_row(300) == 1
    assert oracle.lfg_default_row(1000) == 2
    assert oracle.lfg_default_row(4096) == 5
    assert oracle.lfg_default_row(10**6) == 9
    assert oracle.lfg_default_row(10**8) == 9


# ------------------------------------------------------------- conversions
def test_uniform_conversions_ranges():
    """Algorithm 1's conversion: u = mult * raw with mult = 2^-32 lies in [0, 1]
    (1.0 from raw >= 2^32-128 after rounding); the Box-Muller map is open."""
    assert oracle.u01_f32(0) == 0.0
    assert oracle.u01_f32(2**32 - 1) == 1.0
    assert oracle.u01_f32(2**31) == 0.5
    assert oracle.open01(0) == 2.0**-24
    assert oracle.open01(2**32 - 1) == 1.0 - 2.0**-24
    assert np.float32(oracle.open01(123456789)) == oracle.open01(123456789)
    am = float(np.float32(1.0 / M1))
    assert oracle.ran2_u01_f32(1) == np.float32(am)
    assert oracle.ran2_u01_f32(M1 - 1) <= np.nextafter(np.float32(1), np.float32(0))


def test_box_muller_structure():
    """Box-Muller (Sec. II.A): g1^2 + g2^2 = -2 ln u1 and atan2(g2, g1) = 2 pi u2."""
    rng = np.random.default_rng(1)
    for u1, u2 in rng.random((200, 2)):
        g1, g2 = oracle.box_muller_f64(u1, u2)
        assert math.isclose(g1 * g1 + g2 * g2, -2 * math.log(u1), rel_tol=1e-12)
        ang = math.atan2(g2, g1) % (2 * math.pi)
        assert math.isclose(ang, 2 * math.pi * u2, rel_tol=1e-9, abs_tol=1e-9)
        f1, f2 = oracle.box_muller_f32(np.float32(u1), np.float32(u2))
        e1, e2 = oracle.box_muller_f64(float(np.float32(u1)), float(np.float32(u2)))
        assert abs(f1 - e1) <= 4e-7 * abs(e1) + 1e-7 and abs(f2 - e2) <= 4e-7 * abs(e2) + 1e-7


# --------------------------------------------------- statistics (all kinds)
@pytest.mark.parametrize("kind", ["taus", "ran2", "lagfib"])
def test_uniform_statistics(kind):
    """Uniform moments 1/2 and 1/12, 256-bin chi-square and lag-1
    autocorrelation of 2^20 numbers (4-sigma bounds)."""
    g = oracle.Gen(kind, 2024, 4096)
    u = g.fill_uniform(2**20).astype(np.float64)
    n = u.size
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 4 * math.sqrt(1 / 180 / n)
    counts = np.bincount(np.minimum((u * 256).astype(int), 255), minlength=256)
    chi2 = ((counts - n / 256) ** 2 / (n / 256)).sum()
    assert chi2 < 255 + 4 * math.sqrt(2 * 255)
    c = u - 0.5
    r1 = (c[:-1] * c[1:]).mean() / (1 / 12)
    assert abs(r1) < 4 / math.sqrt(n)


@pytest.mark.parametrize("kind", ["taus", "ran2", "lagfib"])
def test_normal_statistics(kind):
    """Box-Muller normals: mean 0, variance 1, kurtosis 3, and a KS test."""
    stats = pytest.importorskip("scipy.stats")
    g = oracle.Gen(kind, 77, 1024)
    z = g.fill_normal(2**20).astype(np.float64)
    n = z.size
    assert abs(z.mean()) < 4 / math.sqrt(n)
    assert abs(z.var() - 1) < 4 * math.sqrt(2 / n)
    k = ((z - z.mean()) ** 4).mean() / z.var() ** 2
    assert abs(k - 3) < 4 * math.sqrt(24 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_fill_layout_per_thread():
    """Fill layout: out[d*S + s] is the d-th draw of stream s; a ragged tail
    draws once more from the first streams only."""
    S = 5
    a = oracle.Gen("taus", 3, S)
    out = a.fill_u32(13)
    c = oracle.Gen("taus", 3, S)
    streams = [[oracle.taus_next(c.state[s]) for _ in range(3)] for s in range(S)]
    exp = [streams[s][d] for idx in range(13) for d, s in [divmod(idx, S)]]
    assert [int(v) for v in out] == exp
    assert np.array_equal(a.state[:3], c.state[:3])          # drew 3 times
    assert not np.array_equal(a.state[3:], c.state[3:])      # drew 2 times


@pytest.mark.parametrize("kind", ["taus", "ran2"])
def test_seed_selected_streams(kind):
    """Seeding a list of stream indices gives the rows a full seeding gives."""
    full = oracle.Gen(kind, 17, 300)
    idx = [0, 5, 299, 123]
    sub = oracle.Gen.streams(kind, 17, idx)
    assert np.array_equal(sub.state, full.state[idx])
