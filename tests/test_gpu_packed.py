"""GPU parity of the packed column-major comparison layout (Sec. III-A).

The packed array is filled from a tiled handle, one op is applied to it
through the C ABI, and the result is copied back and compared with the
oracle; the raw packed array itself is compared with the oracle's
definition of the layout.  Tolerances as in test_gpu_parity.
"""
import numpy as np
import pytest

from oracle import dense as D
from oracle import packed as PK
from workloads import synth as S

pytestmark = pytest.mark.gpu

ok = pytest.importorskip("paper_2604_15765_gb300.orkan")
torch = pytest.importorskip("torch")

TOL = {"c128": 1e-12, "df64": 1e-12, "c64": 1e-5}
DT = {"c128": 0, "c64": 1, "df64": 2}
HAD = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2)
CNOT = np.eye(4, dtype=np.complex128)[[0, 3, 2, 1]]
SWAP = np.eye(4, dtype=np.complex128)[[0, 2, 1, 3]]
ISWAP = np.array([[1, 0, 0, 0], [0, 0, 1j, 0], [0, 1j, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def _tol(dtype, ref):
    scale = float(np.max(np.abs(ref)))
    return TOL[dtype] * (scale if dtype == "c64" else max(1.0, scale))


def _ops(n, rng):
    """(name, packed call, oracle Kraus set, qubits, exact) for every class."""
    out = []
    for q in range(n):
        U = S.haar_unitary(rng, 2)
        out.append(("u1", "unitary", [U], [q], False))
        out.append(("x", "unitary", [D.X], [q], True))
        out.append(("h", "unitary", [HAD], [q], False))
        out.append(("depol", "depol", D.depolarizing_kraus(0.1), [q], False))
        out.append(("ampdamp", "kraus", D.amplitude_damping_kraus(0.05), [q], False))
        ks = [0.4 * (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) for _ in range(3)]
        out.append(("kraus1", "kraus", ks, [q], False))
    if n >= 2:
        pairs = {(0, n - 1), (n - 1, 0)} | {(q, q + 1) for q in range(n - 1)} | {(q + 1, q) for q in range(0, n - 1, 2)}
        for a, b in sorted(pairs):
            out.append(("u2", "unitary", [S.haar_unitary(rng, 4)], [a, b], False))
            for name, G in (("cnot", CNOT), ("swap", SWAP), ("iswap", ISWAP)):
                out.append((name, "unitary", [G], [a, b], True))
    return out


def _apply_packed(buf, n, dtype, call, kraus, qubits, picture, stream):
    pic = ok.ORKAN_STATE if picture == "schrodinger" else ok.ORKAN_OBSERVABLE
    if call == "unitary":
        ok.orkan_packed_apply_unitary(buf.data_ptr(), n, DT[dtype], qubits, kraus[0], pic, stream)
    elif call == "depol":
        ok.orkan_packed_depolarize(buf.data_ptr(), n, DT[dtype], qubits[0], 0.1, stream)
    else:
        ok.orkan_packed_apply_kraus(buf.data_ptr(), n, DT[dtype], qubits, np.array(kraus), pic, stream)


@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
@pytest.mark.parametrize("picture", ["schrodinger", "heisenberg"])
@pytest.mark.parametrize("n,m", [(1, 5), (2, 5), (3, 3), (5, 5), (7, 3), (9, 4)])
def test_packed_single_ops(n, m, dtype, picture):
    rng = S.rng_for(8000 + 13 * n + m)
    N = 1 << n
    H0 = S.ginibre_state(rng, N) if picture == "schrodinger" else S.random_hermitian(rng, N)
    stream = torch.cuda.current_stream().cuda_stream
    h = ok.orkan_alloc(n, DT[dtype], m)
    buf = torch.empty(ok.orkan_packed_bytes(n, DT[dtype]), dtype=torch.uint8, device="cuda")
    try:
        ok.orkan_set_stream(h, stream)
        for name, call, kraus, qubits, exact in _ops(n, rng):
            ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H0)
            if picture == "heisenberg":
                ok.orkan_set_picture(h, ok.ORKAN_OBSERVABLE)
            before = ok.orkan_to_dense(h)
            ok.orkan_packed_from_tiled(h, buf.data_ptr())
            _apply_packed(buf, n, dtype, call, kraus, qubits, picture, stream)
            ok.orkan_packed_to_tiled(h, buf.data_ptr())
            got = ok.orkan_to_dense(h)
            if exact:
                ref = D.apply_kraus(before, kraus, qubits, picture)
                assert np.array_equal(got, ref), (name, qubits)
            else:
                ref = D.apply_kraus(H0, kraus, qubits, picture)
                err = float(np.max(np.abs(got - ref)))
                assert err <= _tol(dtype, ref), f"{name} on {qubits}: {err:.3e}"
    finally:
        ok.orkan_free(h)


@pytest.mark.parametrize("n", [1, 4, 6])
def test_packed_array_is_the_papers_layout(n):
    """The raw packed array holds H's lower triangle column by column (c128,
    exact), and the round trip through it restores the tiled operator."""
    rng = S.rng_for(8100 + n)
    H0 = S.random_hermitian(rng, 1 << n)
    stream = torch.cuda.current_stream().cuda_stream
    h = ok.orkan_alloc(n, DT["c128"], 3)
    buf = torch.empty(ok.orkan_packed_bytes(n, DT["c128"]), dtype=torch.uint8, device="cuda")
    try:
        ok.orkan_set_stream(h, stream)
        ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H0)
        ok.orkan_packed_from_tiled(h, buf.data_ptr())
        torch.cuda.current_stream().synchronize()
        host = buf.cpu().numpy().view(np.complex128)
        assert np.array_equal(host, PK.to_packed(H0))
        ok.orkan_init_state(h, ok.ORKAN_INIT_ZERO)
        ok.orkan_packed_to_tiled(h, buf.data_ptr())
        assert np.array_equal(ok.orkan_to_dense(h), H0)
    finally:
        ok.orkan_free(h)


@pytest.mark.parametrize("dtype", ["df64", "c128", "c64"])
def test_packed_agrees_with_tiled_at_n13(dtype):
    """The paper's benchmark ops (depolarising, X, H, CNOT) on every target
    at n = 13: packed and tiled results agree on sampled elements (bit for bit
    for the permutations)."""
    n = 13
    N = 1 << n
    rng = S.rng_for(8200)
    psi = S.haar_state_vector(rng, N)
    stream = torch.cuda.current_stream().cuda_stream
    ht = ok.orkan_alloc(n, DT[dtype], 5)
    hp = ok.orkan_alloc(n, DT[dtype], 5)
    buf = torch.empty(ok.orkan_packed_bytes(n, DT[dtype]), dtype=torch.uint8, device="cuda")
    try:
        for h in (ht, hp):
            ok.orkan_set_stream(h, stream)
            ok.orkan_set_fusion(h, 1, False)
            ok.orkan_init_state(h, ok.ORKAN_INIT_PURE, psi)
        ok.orkan_packed_from_tiled(hp, buf.data_ptr())
        for q in range(n):
            ok.orkan_depolarize(ht, q, 0.1)
            ok.orkan_packed_depolarize(buf.data_ptr(), n, DT[dtype], q, 0.1, stream)
            ok.orkan_apply_unitary(ht, [q], HAD)
            ok.orkan_packed_apply_unitary(buf.data_ptr(), n, DT[dtype], [q], HAD, ok.ORKAN_STATE, stream)
            ok.orkan_apply_unitary(ht, [q], D.X)
            ok.orkan_packed_apply_unitary(buf.data_ptr(), n, DT[dtype], [q], D.X, ok.ORKAN_STATE, stream)
            ok.orkan_apply_unitary(ht, [q, (q + 5) % n], CNOT)
            ok.orkan_packed_apply_unitary(buf.data_ptr(), n, DT[dtype], [q, (q + 5) % n], CNOT, ok.ORKAN_STATE,
                                          stream)
        ok.orkan_packed_to_tiled(hp, buf.data_ptr())
        rows = np.concatenate([rng.integers(0, N, 4000), np.arange(0, N, 7)])
        cols = np.concatenate([rng.integers(0, N, 4000), np.arange(0, N, 7)])
        a = ok.orkan_get_elements(ht, rows, cols)
        b = ok.orkan_get_elements(hp, rows, cols)
        scale = float(np.max(np.abs(a)))
        assert float(np.max(np.abs(a - b))) <= (1e-12 if dtype != "c64" else 1e-5) * scale
        assert abs(ok.orkan_trace(ht) - ok.orkan_trace(hp)) <= (1e-12 if dtype != "c64" else 1e-5)
    finally:
        ok.orkan_free(ht)
        ok.orkan_free(hp)
