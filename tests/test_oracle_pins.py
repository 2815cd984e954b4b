"""Pins for the CPU oracle: values fixed by the paper or by the mathematics.

Each test checks the oracle against something other than itself: the paper's
Table I, closed forms of the named channels on Bell and GHZ states, brute
force over basis states, independent constructions of the same object, and
the invariants every Kraus map has (hermiticity, trace, positivity, spectrum,
trace duality).  ``test_planted_mistakes_are_caught`` plants typical
mistakes in the oracle and checks that these pins fail.
"""
import itertools
import os

import numpy as np
import pytest

from oracle import dense as D
from oracle import tiled as T
from workloads import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
UNITS = {"B": 1, "KiB": 1 << 10, "MiB": 1 << 20, "GiB": 1 << 30}


def _parse_size(tok):
    for u in ("KiB", "MiB", "GiB", "B"):
        if tok.endswith(u):
            return float(tok[: -len(u)]) * UNITS[u], tok[: -len(u)]
    raise ValueError(tok)


def _round_like(value_bytes, printed):
    """Round value (in the printed unit) to the printed number of decimals."""
    dec = len(printed.split(".")[1]) if "." in printed else 0
    return round(value_bytes, dec)


# ---------------------------------------------------------------- Table I
def test_table1_memory_footprint():
    rows = []
    with open(os.path.join(GOLDEN, "table1_memory_footprint.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    assert len(rows) == 5
    for n_s, full_s, packed_s, tiled_s, ratio_s in rows:
        n = int(n_s)
        N = 1 << n
        full = N * N * 16
        packed = N * (N + 1) // 2 * 16
        tiled = T.stored_bytes(n, 5, 16)
        for val, tok in ((full, full_s), (packed, packed_s), (tiled, tiled_s)):
            expect, printed = _parse_size(tok)
            unit = tok[len(printed):]
            assert _round_like(val / UNITS[unit], printed) == pytest.approx(float(printed)), (n, tok, val)
        dec = len(ratio_s.split(".")[1]) if "." in ratio_s else 0
        assert round(tiled / packed, dec) == pytest.approx(float(ratio_s)), (n, tiled / packed)


def test_storage_formula_and_padding():
    for n in range(1, 12):
        for m in range(0, 7):
            N, M = 1 << n, 1 << m
            expect = M * M if N < M else N * (N + M) // 2
            assert T.stored_elements(n, m) == expect


# ---------------------------------------------------------------- layout
@pytest.mark.parametrize("n,m", [(1, 5), (2, 5), (3, 1), (4, 2), (5, 5), (6, 3), (6, 0), (7, 2)])
def test_tiled_roundtrip_and_element_map(n, m):
    rng = S.rng_for(11 + n + 10 * m)
    H = S.random_hermitian(rng, 1 << n)
    buf = T.to_tiled(H, m)
    assert buf.size == T.stored_elements(n, m)
    assert np.array_equal(T.from_tiled(buf, n, m), H)
    N = 1 << n
    for i in range(N):
        for j in range(N):
            off, conj = T.element_offset(i, j, n, m)
            v = np.conj(buf[off]) if conj else buf[off]
            assert v == H[i, j]


def test_m0_is_row_major_packed():
    """Footnote of Sec. IV-A: m = 0 recovers the packed format up to order."""
    rng = S.rng_for(5)
    n = 5
    H = S.random_hermitian(rng, 1 << n)
    packed_rows = np.concatenate([H[i, : i + 1] for i in range(1 << n)])
    assert np.array_equal(T.to_tiled(H, 0), packed_rows)


def _extract(g, A):
    return sum(((g >> p) & 1) << l for l, p in enumerate(sorted(A)))


def _compress(g, A, n):
    rest = [p for p in range(n) if p not in A]
    return sum(((g >> p) & 1) << l for l, p in enumerate(rest))


def test_insert_bits_bruteforce():
    """Subroutine 1: inserting the bits of a at A into s reproduces every
    global index, for all subsets A of size 1..3 of n <= 6 bits."""
    for n in range(1, 7):
        for k in range(1, min(3, n) + 1):
            for A in itertools.combinations(range(n), k):
                for g in range(1 << n):
                    assert T.insert_bits(_compress(g, A, n), _extract(g, A), A) == g


# ---------------------------------------------------------------- embedding
def _embed_by_definition(L, qubits, n):
    """K[i, j] = L[a(i), a(j)] if i and j agree outside ``qubits`` else 0,
    with a(i) the local index whose bit l is bit qubits[l] of i."""
    N = 1 << n
    K = np.zeros((N, N), dtype=np.complex128)
    mask = sum(1 << q for q in qubits)
    for i in range(N):
        ai = sum(((i >> q) & 1) << l for l, q in enumerate(qubits))
        for j in range(N):
            if (i & ~mask) == (j & ~mask):
                aj = sum(((j >> q) & 1) << l for l, q in enumerate(qubits))
                K[i, j] = L[ai, aj]
    return K


def test_embed_matches_definition():
    rng = S.rng_for(7)
    n = 4
    for k in (1, 2, 3):
        for qubits in itertools.permutations(range(n), k):
            L = rng.standard_normal((1 << k, 1 << k)) + 1j * rng.standard_normal((1 << k, 1 << k))
            assert np.array_equal(D.embed(L, qubits, n, sparse=False), _embed_by_definition(L, list(qubits), n))


def test_dense_and_sparse_embeddings_agree():
    rng = S.rng_for(8)
    for n in (3, 5, 6):
        for qubits in ([0], [n - 1], [1, n - 1], [n - 1, 0], [2, 1]):
            L = S.haar_unitary(rng, 1 << len(qubits))
            Kd = D.embed(L, qubits, n, sparse=False)
            Ks = D.embed(L, qubits, n, sparse=True).toarray()
            assert np.array_equal(Kd, Ks)


def test_sparse_apply_matches_dense_apply(monkeypatch):
    rng = S.rng_for(9)
    n = 6
    rho = S.ginibre_state(rng, 1 << n)
    U = S.haar_unitary(rng, 4)
    dense = D.apply_unitary(rho, U, [1, 4])
    monkeypatch.setattr(D, "DENSE_MAX_N", 2)
    sparse = D.apply_unitary(rho, U, [1, 4])
    assert np.max(np.abs(dense - sparse)) < 1e-15


def test_cnot_on_basis_states():
    """Bit l of a 2-qubit matrix's index is qubits[l]: CNOT with its control
    on index bit 0 flips qubit qubits[1] exactly when qubit qubits[0] is 1."""
    cnot = np.zeros((4, 4), dtype=np.complex128)
    for b in range(4):
        b0, b1 = b & 1, (b >> 1) & 1
        cnot[((b1 ^ b0) << 1) | b0, b] = 1
    n = 4
    for c, t in itertools.permutations(range(n), 2):
        for x in range(1 << n):
            rho = np.zeros((1 << n, 1 << n), dtype=np.complex128)
            rho[x, x] = 1
            out = D.apply_unitary(rho, cnot, [c, t])
            y = x ^ (((x >> c) & 1) << t)
            expect = np.zeros_like(rho)
            expect[y, y] = 1
            assert np.array_equal(out, expect)


def test_pauli_x_is_a_pure_swap():
    """Sec. II-B: X on qubit a swaps h[i,j] with h[i^2^a, j^2^a], bit for bit."""
    rng = S.rng_for(10)
    n = 5
    H = S.random_hermitian(rng, 1 << n)
    for a in range(n):
        perm = np.arange(1 << n) ^ (1 << a)
        assert np.array_equal(D.apply_unitary(H, D.X, [a]), H[np.ix_(perm, perm)])


# ---------------------------------------------------------------- channels
def _depolarizing_closed_form(rho, q, p):
    """(1 - l) rho + l (I/2 (x)_q tr_q rho) with l = 4p/3, built elementwise."""
    lam = 4.0 * p / 3.0
    N = rho.shape[0]
    out = (1 - lam) * rho.copy()
    bit = 1 << q
    for i in range(N):
        for j in range(N):
            if ((i ^ j) & bit) == 0:
                i0, j0 = i & ~bit, j & ~bit
                out[i, j] += lam * 0.5 * (rho[i0, j0] + rho[i0 | bit, j0 | bit])
    return out


def test_depolarizing_closed_form():
    rng = S.rng_for(12)
    n = 4
    rho = S.ginibre_state(rng, 1 << n)
    for q in range(n):
        for p in (0.0, 0.01, 0.1, 0.75):
            got = D.depolarize(rho, q, p)
            assert np.max(np.abs(got - _depolarizing_closed_form(rho, q, p))) < 1e-15


def _bell():
    v = np.zeros(4, dtype=np.complex128)
    v[0] = v[3] = 1 / np.sqrt(2)
    return np.outer(v, v.conj())


def test_bell_depolarized_is_werner():
    for q in (0, 1):
        for p in (0.03, 0.1, 0.4):
            lam = 4 * p / 3
            rho = D.depolarize(_bell(), q, p)
            werner = (1 - lam) * _bell() + lam * np.eye(4) / 4
            assert np.max(np.abs(rho - werner)) < 1e-15
            assert D.expect_pauli(rho, "XX") == pytest.approx(1 - lam, abs=1e-15)
            assert D.expect_pauli(rho, "ZZ") == pytest.approx(1 - lam, abs=1e-15)
            assert D.expect_pauli(rho, "YY") == pytest.approx(-(1 - lam), abs=1e-15)


def test_bell_amplitude_damping():
    for g in (0.0, 0.05, 0.3, 1.0):
        rho = D.amplitude_damp(_bell(), 0, g)
        expect = np.zeros((4, 4), dtype=np.complex128)
        expect[0, 0] = 0.5
        expect[2, 2] = g / 2
        expect[3, 3] = (1 - g) / 2
        expect[0, 3] = expect[3, 0] = np.sqrt(1 - g) / 2
        assert np.max(np.abs(rho - expect)) <= 2.3e-16   # two roundings of 0.5-sized values


def test_ghz_depolarized():
    n = 5
    N = 1 << n
    v = np.zeros(N, dtype=np.complex128)
    v[0] = v[-1] = 1 / np.sqrt(2)
    ghz = np.outer(v, v.conj())
    p = 0.12
    lam = 4 * p / 3
    for q in range(n):
        rho = D.depolarize(ghz, q, p)
        assert rho[0, 0].real == pytest.approx(0.5 - lam / 4, abs=1e-15)
        assert rho[N - 1, N - 1].real == pytest.approx(0.5 - lam / 4, abs=1e-15)
        assert rho[1 << q, 1 << q].real == pytest.approx(lam / 4, abs=1e-15)
        assert rho[(N - 1) ^ (1 << q), (N - 1) ^ (1 << q)].real == pytest.approx(lam / 4, abs=1e-15)
        assert rho[0, N - 1].real == pytest.approx((1 - lam) / 2, abs=1e-15)
        others = np.abs(rho).copy()
        for (i, j) in [(0, 0), (N - 1, N - 1), (1 << q, 1 << q),
                       ((N - 1) ^ (1 << q), (N - 1) ^ (1 << q)), (0, N - 1), (N - 1, 0)]:
            others[i, j] = 0
        assert others.max() < 1e-16


def test_dephasing_closed_form():
    """Dephasing p multiplies every coherence across qubit q by (1 - 2p)."""
    rng = S.rng_for(13)
    n = 3
    rho = S.ginibre_state(rng, 1 << n)
    for q in range(n):
        got = D.dephase(rho, q, 0.2)
        N = 1 << n
        fac = np.array([[1.0 if ((i ^ j) >> q) & 1 == 0 else 0.6 for j in range(N)] for i in range(N)])
        assert np.max(np.abs(got - rho * fac)) < 1e-15


# ---------------------------------------------------------------- invariants
def test_invariants_on_random_circuits():
    for seed in range(3):
        rng = S.rng_for(100 + seed)
        n = 4
        rho = S.ginibre_state(rng, 1 << n)
        ops = S.random_mixed_circuit(rng, n, 40)
        for op in ops:
            before = rho
            rho, _ = D.apply_op(rho, op)
            assert np.max(np.abs(rho - rho.conj().T)) < 1e-14
            assert abs(np.trace(rho) - 1) < 1e-13
            ev = np.linalg.eigvalsh(0.5 * (rho + rho.conj().T))
            assert ev.min() > -1e-13
            if op["kind"] == "unitary":
                e0 = np.linalg.eigvalsh(0.5 * (before + before.conj().T))
                assert np.max(np.abs(ev - e0)) < 1e-13


def test_trace_duality():
    """tr(O Phi(rho)) = tr(Phi*(O) rho) for a 20-op circuit (Sec. I, Sec. II)."""
    for seed in range(3):
        rng = S.rng_for(200 + seed)
        n = 4
        rho = S.ginibre_state(rng, 1 << n)
        strings, coeffs = S.random_pauli_sum(rng, n, 16)
        O = D.pauli_sum(strings, coeffs)
        ops = S.random_mixed_circuit(rng, n, 20, with_measure=False)
        rho_t, _ = D.run_circuit(rho, ops, "schrodinger")
        O_t, _ = D.run_circuit(O, list(reversed(ops)), "heisenberg")
        assert D.expect(rho_t, O) == pytest.approx(D.expect(rho, O_t), abs=1e-12)


def test_heisenberg_of_hadamard():
    Hd = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2)
    assert np.max(np.abs(D.apply_unitary(D.Z, Hd, [0], "heisenberg") - D.X)) < 1e-15
    # Heisenberg of amplitude damping on Z: K0^+ Z K0 + K1^+ Z K1 = diag(1, 1-2g)... = (g) I + (1-g) Z
    g = 0.3
    got = D.amplitude_damp(D.Z, 0, g, "heisenberg")
    assert np.max(np.abs(got - (g * np.eye(2) + (1 - g) * D.Z))) < 1e-15


# ---------------------------------------------------------------- measurement
def test_measurement_probabilities_and_repeat():
    rng = S.rng_for(300)
    n = 4
    rho = S.ginibre_state(rng, 1 << n)
    for q in range(n):
        p0, p1 = D.born_probabilities(rho, q)
        assert p0 + p1 == pytest.approx(np.trace(rho).real, abs=1e-14)
        diag = np.real(np.diag(rho))
        assert p0 == pytest.approx(sum(diag[i] for i in range(1 << n) if not (i >> q) & 1), abs=1e-15)
        for u in (0.1, 0.9):
            post, b, pb = D.measure(rho, q, u)
            assert b == (0 if u < p0 else 1)
            assert np.trace(post).real == pytest.approx(1.0, abs=1e-14)
            again, b2, pb2 = D.measure(post, q, 0.5)
            assert b2 == b and pb2 == pytest.approx(1.0, abs=1e-14)
            for i in range(1 << n):
                for j in range(1 << n):
                    if ((i >> q) & 1) != b or ((j >> q) & 1) != b:
                        assert post[i, j] == 0


# ---------------------------------------------------------------- readouts
def test_pauli_expectations_on_basis_and_ghz():
    n = 4
    for x in range(1 << n):
        rho = np.zeros((1 << n, 1 << n), dtype=np.complex128)
        rho[x, x] = 1
        for l in range(n):
            s = ["I"] * n
            s[l] = "Z"
            assert D.expect_pauli(rho, "".join(s)) == (-1) ** ((x >> l) & 1)
            s[l] = "X"
            assert D.expect_pauli(rho, "".join(s)) == 0
    v = np.zeros(1 << n, dtype=np.complex128)
    v[0] = v[-1] = 1 / np.sqrt(2)
    ghz = np.outer(v, v.conj())
    assert D.expect_pauli(ghz, "X" * n) == pytest.approx(1.0)
    assert D.expect_pauli(ghz, "ZZII") == pytest.approx(1.0)
    assert D.expect_pauli(_bell(), "YY") == pytest.approx(-1.0)
    assert D.expect_pauli(np.eye(1 << n) / (1 << n), "XYZI") == 0


def test_pauli_y_eigenstate():
    """|+i> = (|0> + i|1>)/sqrt2 has <Y> = +1; on qubit 1 of a 2-qubit
    product with |0> on qubit 0, <ZY> (char 0 = Z on qubit 0) = +1."""
    v = np.array([1, 1j]) / np.sqrt(2)
    assert D.expect_pauli(np.outer(v, v.conj()), "Y") == pytest.approx(1.0)
    w = np.kron(v, np.array([1, 0]))   # qubit 1 in |+i>, qubit 0 in |0>
    rho = np.outer(w, w.conj())
    assert D.expect_pauli(rho, "ZY") == pytest.approx(1.0)
    assert D.expect_pauli(rho, "YZ") == pytest.approx(0.0)


_SIGMA = {
    "I": ((1, 0), (0, 1)),
    "X": ((0, 1), (1, 0)),
    "Y": ((0, -1j), (1j, 0)),
    "Z": ((1, 0), (0, -1)),
}


def _pauli_element(pauli, i, j):
    """<i|P|j> = prod_l sigma_{pauli[l]}[bit l of i, bit l of j], from the
    definition of a tensor product of single-qubit Paulis (character l on
    qubit l), without any Kronecker product."""
    v = 1.0 + 0j
    for l, ch in enumerate(pauli):
        v *= _SIGMA[ch][(i >> l) & 1][(j >> l) & 1]
    return v


def test_pauli_sum_coefficients():
    """O = sum_a c_a P_a (the observable of the Heisenberg workloads): the
    Pauli strings are orthogonal, tr(P_a P_b) = N delta_ab, so
    tr(P_a O) / N = c_a for distinct strings and 0 for a string not in the
    sum.  A single term c P has the eigenvalues +c and -c, N / 2 times each."""
    rng = S.rng_for(410)
    n = 3
    N = 1 << n
    strings = ["XIZ", "YYI", "IZX", "ZXY", "III"]
    coeffs = rng.standard_normal(len(strings))
    O = D.pauli_sum(strings, coeffs)
    for s, c in list(zip(strings, coeffs)) + [("XXX", 0.0), ("IIZ", 0.0)]:
        tr = sum(_pauli_element(s, j, i) * O[i, j] for i in range(N) for j in range(N))
        assert tr / N == pytest.approx(c, abs=1e-13)
    for s in ("XIZ", "ZYX", "IIY"):
        ev = np.sort(np.linalg.eigvalsh(D.pauli_sum([s], [-1.75])))
        assert np.max(np.abs(ev - np.repeat([-1.75, 1.75], N // 2))) < 1e-14


def test_project_keeps_only_the_outcome_block():
    """Pi_b H Pi_b (Sec. II, a trace non-increasing map): every element whose
    row or column has bit q != b becomes 0, the rest are unchanged; a state
    with qubit q in |b'> projects to 0 for b' != b and is left as it is for
    b' = b; and measure() equals project() divided by p_b."""
    rng = S.rng_for(420)
    n = 3
    N = 1 << n
    H = S.random_hermitian(rng, N)
    for q in range(n):
        for b in (0, 1):
            got = D.project(H, q, b)
            for i in range(N):
                for j in range(N):
                    keep = ((i >> q) & 1) == b and ((j >> q) & 1) == b
                    assert got[i, j] == (H[i, j] if keep else 0)
    rest = S.ginibre_state(rng, 1 << (n - 1))
    for q in range(n):
        for bp in (0, 1):
            e = np.zeros((2, 2), dtype=np.complex128)
            e[bp, bp] = 1
            # qubit q in |bp>, the other qubits in the state ``rest``
            full = np.zeros((N, N), dtype=np.complex128)
            others = [x for x in range(n) if x != q]
            for i in range(N):
                for j in range(N):
                    ri = sum(((i >> x) & 1) << t for t, x in enumerate(others))
                    rj = sum(((j >> x) & 1) << t for t, x in enumerate(others))
                    full[i, j] = e[(i >> q) & 1, (j >> q) & 1] * rest[ri, rj]
            for b in (0, 1):
                got = D.project(full, q, b)
                if b == bp:
                    assert np.array_equal(got, full)
                else:
                    assert not np.any(got)
    rho = S.ginibre_state(rng, N)
    for q in range(n):
        for u in (0.2, 0.8):
            post, b, _ = D.measure(rho, q, u)
            pb = D.born_probabilities(rho, q)[b]
            assert np.max(np.abs(post - D.project(rho, q, b) / pb)) < 1e-15


def test_tiled_mean_value_equals_trace():
    rng = S.rng_for(400)
    for n, m in ((3, 1), (5, 2), (6, 5), (2, 5), (6, 3)):
        rho = S.ginibre_state(rng, 1 << n)
        O = S.random_hermitian(rng, 1 << n)
        got = T.tiled_mean_value(T.to_tiled(rho, m), T.to_tiled(O, m), n, m)
        assert got == pytest.approx(np.trace(rho @ O).real, abs=1e-13)


def test_trace_distance_closed_form():
    a = np.diag([1.0, 0.0]).astype(np.complex128)
    b = np.diag([0.0, 1.0]).astype(np.complex128)
    assert D.trace_distance(a, b) == pytest.approx(1.0)
    assert D.trace_distance(a, 0.5 * np.eye(2)) == pytest.approx(0.5)


# ---------------------------------------------------------------- teeth
def test_planted_mistakes_are_caught(monkeypatch):
    """Plant typical oracle mistakes on the CPU and check a pin fails."""
    # 1) a dropped conjugate: K H K^T instead of K H K^dagger
    def bad_conj(K, H):
        KH = D._left(K, H)
        return D._left(K, KH.T).T
    with monkeypatch.context() as mp:
        mp.setattr(D, "_conjugate", bad_conj)
        with pytest.raises(AssertionError):
            test_bell_depolarized_is_werner()
    # 2) a dropped Kraus term
    orig = D.depolarizing_kraus
    with monkeypatch.context() as mp:
        mp.setattr(D, "depolarizing_kraus", lambda p: orig(p)[:3])
        with pytest.raises(AssertionError):
            test_depolarizing_closed_form()
    # 3) a transposed operator in the embedding
    orig_embed = D.embed
    with monkeypatch.context() as mp:
        mp.setattr(D, "embed", lambda L, q, n, sparse=None: orig_embed(np.asarray(L).T, q, n, sparse))
        with pytest.raises(AssertionError):
            test_bell_amplitude_damping()
    # 4) a wrong sign in Y
    with monkeypatch.context() as mp:
        mp.setattr(D, "PAULI", dict(D.PAULI, Y=-D.Y))
        with pytest.raises(AssertionError):
            test_pauli_y_eigenstate()
    # 5) swapped qubit order in the Kronecker product
    with monkeypatch.context() as mp:
        mp.setattr(D, "embed", lambda L, q, n, sparse=None: orig_embed(L, [n - 1 - x for x in q], n, sparse))
        with pytest.raises(AssertionError):
            test_bell_amplitude_damping()
    # 6) swapped coefficients in the Pauli sum
    orig_sum = D.pauli_sum
    with monkeypatch.context() as mp:
        mp.setattr(D, "pauli_sum", lambda s, c: orig_sum(s, list(c)[::-1]))
        with pytest.raises(AssertionError):
            test_pauli_sum_coefficients()
    # 7) a dropped term in the Pauli sum
    with monkeypatch.context() as mp:
        mp.setattr(D, "pauli_sum", lambda s, c: orig_sum(s[:-1], list(c)[:-1]))
        with pytest.raises(AssertionError):
            test_pauli_sum_coefficients()
    # 8) the projector onto the other outcome
    orig_proj = D.projector
    with monkeypatch.context() as mp:
        mp.setattr(D, "project", lambda H, q, b: D.apply_kraus(H, [orig_proj(1 - b)], [q]))
        with pytest.raises(AssertionError):
            test_project_keeps_only_the_outcome_block()


def test_factored_kraus_matches_dense():
    """Eq. (1) on H = sum_v v v^dagger through the factors equals the dense map,
    and factored_elements reads H's entries (used for sampled checks at large n)."""
    rng = S.rng_for(600)
    n = 5
    vecs = [S.haar_state_vector(rng, 1 << n) * w for w in (0.7, 0.5, 0.2)]
    H = sum(np.outer(v, v.conj()) for v in vecs)
    for kraus, qubits in ((D.depolarizing_kraus(0.2), [3]), ([S.haar_unitary(rng, 4)], [4, 1]),
                          (D.amplitude_damping_kraus(0.3), [0])):
        out = D.apply_kraus_to_factors(vecs, kraus, qubits, n)
        dense = sum(np.outer(v, v.conj()) for v in out)
        assert np.max(np.abs(dense - D.apply_kraus(H, kraus, qubits))) < 1e-15
        rows, cols = rng.integers(0, 1 << n, 50), rng.integers(0, 1 << n, 50)
        assert np.max(np.abs(D.factored_elements(out, rows, cols) - dense[rows, cols])) < 1e-15


# ---------------------------------------------------------------- k = 3
def _toffoli():
    """Controls on index bits 0 and 1, target on bit 2."""
    T = np.zeros((8, 8), dtype=np.complex128)
    for b in range(8):
        T[b ^ (4 if (b & 3) == 3 else 0), b] = 1
    return T


def test_toffoli_on_basis_states():
    """A 3-qubit gate with unsorted qubits: Toffoli flips qubits[2] exactly
    when qubits[0] and qubits[1] are both 1, for every ordered triple."""
    n = 4
    T = _toffoli()
    for c0, c1, t in itertools.permutations(range(n), 3):
        for x in range(1 << n):
            rho = np.zeros((1 << n, 1 << n), dtype=np.complex128)
            rho[x, x] = 1
            y = x ^ ((((x >> c0) & 1) & ((x >> c1) & 1)) << t)
            expect = np.zeros_like(rho)
            expect[y, y] = 1
            assert np.array_equal(D.apply_unitary(rho, T, [c0, c1, t]), expect)


def test_three_qubit_product_equals_single_qubit_gates():
    """kron(U2, U1, U0) on qubits [a, b, c] (bit l <-> qubits[l]) equals U0 on
    a, U1 on b and U2 on c applied one at a time; the single-qubit embeddings
    are plain Kronecker products with no permutation."""
    rng = S.rng_for(610)
    n = 5
    rho = S.ginibre_state(rng, 1 << n)
    for qubits in ([4, 0, 2], [1, 3, 0], [0, 1, 2], [2, 4, 3]):
        us = [S.haar_unitary(rng, 2) for _ in range(3)]
        L = np.kron(us[2], np.kron(us[1], us[0]))
        seq = rho
        for u, q in zip(us, qubits):
            seq = D.apply_unitary(seq, u, [q])
        assert np.max(np.abs(D.apply_unitary(rho, L, qubits) - seq)) < 1e-15


# ---------------------------------------------------------------- packed layout
def test_packed_layout_by_enumeration():
    """Sec. III-A: walking the lower triangle column by column visits the
    offsets 0, 1, 2, ... of the closed form; the storage is N (N + 1) / 2
    elements (Table I's packed column)."""
    from oracle import packed as PK
    for n in range(1, 7):
        N = 1 << n
        pos = 0
        for j in range(N):
            for i in range(j, N):
                assert PK.packed_offset(i, j, n) == (pos, False)
                assert PK.packed_offset(j, i, n) == (pos, i != j)
                pos += 1
        assert pos == PK.packed_elements(n) == N * (N + 1) // 2
    rng = S.rng_for(620)
    H = S.random_hermitian(rng, 16)
    buf = PK.to_packed(H)
    assert buf.size == PK.packed_elements(4)
    assert np.array_equal(PK.from_packed(buf, 4), H)
    for i, j in [(3, 1), (1, 3), (15, 0), (0, 15), (7, 7)]:
        off, cj = PK.packed_offset(i, j, 4)
        assert (np.conj(buf[off]) if cj else buf[off]) == H[i, j]
