"""Pins of the CPU oracle against things other than itself (CPU only).

Each test checks the oracle against a closed form, an independent brute-force
construction (Kronecker products, explicit bit-permutation matrices), a textbook
special case or a value printed in the paper (tests/golden/paper_values.txt), so
that a dropped term, a wrong sign or index, or a transposed operand in the oracle
fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from tests.conftest import load_golden

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

I2 = np.eye(2, dtype=np.complex128)
P0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)
P1 = np.array([[0, 0], [0, 1]], dtype=np.complex128)


def haar(d, rng):
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / math.sqrt(2)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def kron_list(mats_by_qubit, n):
    """Kronecker product with qubit n-1 as the leftmost factor (index bit q = qubit q)."""
    out = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        out = np.kron(out, mats_by_qubit.get(q, I2))
    return out


def bit_perm_matrix(n, dest):
    """P|i> = |j> where bit b of i moves to bit dest[b] of j."""
    d = 1 << n
    P = np.zeros((d, d))
    for i in range(d):
        j = 0
        for b in range(n):
            j |= ((i >> b) & 1) << dest[b]
        P[j, i] = 1
    return P


def rand_state(n, seed):
    return workloads.random_state(n, seed)


# -- gates ---------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 3, 5])
def test_single_qubit_gate_matches_kronecker(n):
    rng = np.random.default_rng(10 + n)
    for q in range(n):
        U = haar(2, rng)
        psi = rand_state(n, 100 + q)
        st = oracle.OracleState(n, psi=psi)
        st.apply_matrix(U, [q])
        np.testing.assert_allclose(st.psi, kron_list({q: U}, n) @ psi, atol=1e-13)


@pytest.mark.parametrize("controls,target", [((0,), 1), ((2,), 0), ((1, 3), 2), ((4, 0, 2), 3)])
def test_controlled_gate_matches_projector_sum(controls, target):
    n = 5
    rng = np.random.default_rng(7)
    U = haar(2, rng)
    all1 = {c: P1 for c in controls}
    full = np.eye(1 << n) - kron_list(all1, n) + kron_list({**all1, target: U}, n)
    psi = rand_state(n, 3)
    st = oracle.OracleState(n, psi=psi)
    st.apply_matrix(U, [target], controls)
    np.testing.assert_allclose(st.psi, full @ psi, atol=1e-13)


@pytest.mark.parametrize("targets", [(0, 1), (1, 0), (4, 1), (2, 5, 0), (5, 3, 1, 4)])
def test_k_qubit_gate_on_arbitrary_targets(targets):
    n, k = 6, len(targets)
    rng = np.random.default_rng(sum(targets) + 31 * k)
    U = haar(1 << k, rng)
    # U acts on the top k index bits (its row MSB = bit n-1); move bit n-1-a to targets[a].
    rest = [q for q in range(n) if q not in targets]
    dest = {}
    for a in range(k):
        dest[n - 1 - a] = targets[a]
    for b, q in enumerate(rest):
        dest[b] = q
    P = bit_perm_matrix(n, dest)
    full = P @ np.kron(U, np.eye(1 << (n - k))) @ P.T
    psi = rand_state(n, 5)
    st = oracle.OracleState(n, psi=psi)
    st.apply_matrix(U, list(targets))
    np.testing.assert_allclose(st.psi, full @ psi, atol=1e-13)


def test_textbook_special_cases_of_u3_and_phase():
    np.testing.assert_allclose(oracle.u3(math.pi, 0, math.pi), [[0, 1], [1, 0]], atol=1e-15)
    np.testing.assert_allclose(oracle.u3(math.pi / 2, 0, math.pi), np.array([[1, 1], [1, -1]]) / math.sqrt(2),
                               atol=1e-15)
    np.testing.assert_allclose(oracle.u3(0, 0, 0.7), [[1, 0], [0, np.exp(0.7j)]], atol=1e-15)
    np.testing.assert_allclose(oracle.u3(math.pi, math.pi / 2, math.pi / 2), [[0, -1j], [1j, 0]], atol=1e-15)
    for th, ph, la in [(0.3, 1.1, 2.0), (2.9, 4.0, 5.5)]:
        U = oracle.u3(th, ph, la)
        np.testing.assert_allclose(U.conj().T @ U, np.eye(2), atol=1e-15)


def test_named_single_qubit_gates_follow_from_x_and_h():
    """Y, Z, S, S^dagger, T, T^dagger from X and H alone (X and H are pinned by the
    Bell/GHZ states and the U3 special cases): Z = H X H, Y = i X Z, S^2 = Z with
    S X S^dagger = Y (which fixes the sign of S), T^2 = S with T X T^dagger =
    (X + Y)/sqrt(2) (which fixes the sign of T), and the daggers as inverses."""
    X, H = oracle.GATES_1Q["x"], oracle.GATES_1Q["h"]
    Z = H @ X @ H
    Y = 1j * X @ Z
    g = oracle.GATES_1Q
    np.testing.assert_allclose(g["z"], Z, atol=1e-15)
    np.testing.assert_allclose(g["y"], Y, atol=1e-15)
    S, T = g["s"], g["t"]
    for D in (S, T):   # diagonal with D[0, 0] = 1 (a phase gate)
        assert D[0, 1] == 0 and D[1, 0] == 0 and D[0, 0] == 1
    np.testing.assert_allclose(S @ S, Z, atol=1e-15)
    np.testing.assert_allclose(S @ X @ S.conj().T, Y, atol=1e-15)
    np.testing.assert_allclose(g["sdg"] @ S, I2, atol=1e-15)
    np.testing.assert_allclose(T @ T, S, atol=1e-15)
    np.testing.assert_allclose(T @ X @ T.conj().T, (X + Y) / math.sqrt(2), atol=1e-15)
    np.testing.assert_allclose(g["tdg"] @ T, I2, atol=1e-15)


def test_rz_phase_and_u3_against_matrix_exponentials():
    """RZ(t) = exp(-i t Z / 2) and P(t) = exp(i t (I - Z) / 2) by scipy's expm of
    the generators; RZ(t) = e^{-i t/2} P(t); U3(th, ph, la) = e^{i (ph + la)/2}
    RZ(ph) RY(th) RZ(la) with RY(th) = exp(-i th Y / 2) (the OpenQASM 2 identity)."""
    from scipy.linalg import expm

    X, H = oracle.GATES_1Q["x"], oracle.GATES_1Q["h"]
    Z = H @ X @ H
    Y = 1j * X @ Z
    for t in (0.0, 0.3, math.pi / 2, 2.5, math.pi, 5.9):
        np.testing.assert_allclose(oracle.gate_matrix("rz", [t]), expm(-0.5j * t * Z), atol=1e-14)
        np.testing.assert_allclose(oracle.gate_matrix("p", [t]), expm(0.5j * t * (I2 - Z)), atol=1e-14)
        np.testing.assert_allclose(oracle.gate_matrix("rz", [t]), np.exp(-0.5j * t) * oracle.gate_matrix("p", [t]),
                                   atol=1e-15)
    np.testing.assert_allclose(oracle.gate_matrix("p", [math.pi / 2]), oracle.GATES_1Q["s"], atol=1e-15)
    np.testing.assert_allclose(oracle.gate_matrix("p", [math.pi / 4]), oracle.GATES_1Q["t"], atol=1e-15)
    rng = np.random.default_rng(77)
    for th, ph, la in rng.uniform(0, 2 * math.pi, size=(6, 3)):
        want = np.exp(0.5j * (ph + la)) * expm(-0.5j * ph * Z) @ expm(-0.5j * th * Y) @ expm(-0.5j * la * Z)
        np.testing.assert_allclose(oracle.gate_matrix("u3", [th, ph, la]), want, atol=1e-14)


def test_swap_gate_exchanges_qubits():
    n = 4
    psi = rand_state(n, 9)
    st = oracle.OracleState(n, psi=psi)
    st.apply_matrix(oracle.SWAP, [3, 1])
    P = bit_perm_matrix(n, {0: 0, 1: 3, 2: 2, 3: 1})
    np.testing.assert_allclose(st.psi, P @ psi, atol=1e-15)


def test_invalid_arguments_are_rejected():
    st = oracle.OracleState(3)
    with pytest.raises(ValueError):
        st.apply_matrix(oracle.GATES_1Q["h"], [3])
    with pytest.raises(ValueError):
        st.apply_matrix(np.eye(4), [1, 1])
    with pytest.raises(ValueError):
        st.apply_matrix(oracle.GATES_1Q["x"], [0], [0])


# -- composites ------------------------------------------------------------------

def bitrev(x, n):
    return int(format(x, f"0{n}b")[::-1], 2)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_qft_sequence_is_the_dft_closed_form(n):
    """Appendix A's QFT commands (H, CPHASE pi/2^(i+1), end-for-end SWAPs) with
    qubit 0 the register MSB equal F|x> = 2^(-n/2) sum_y e^{2 pi i x y / 2^n}|y>."""
    ops = workloads.qft_ops(range(n))
    d = 1 << n
    for x in range(d):
        psi = np.zeros(d, dtype=np.complex128)
        psi[bitrev(x, n)] = 1.0
        st = oracle.OracleState(n, psi=psi)
        for op in ops:
            st.apply_op(op)
        expect = np.zeros(d, dtype=np.complex128)
        for y in range(d):
            expect[bitrev(y, n)] = np.exp(2j * math.pi * x * y / d) / math.sqrt(d)
        np.testing.assert_allclose(st.psi, expect, atol=1e-13)


def test_qft_gate_counts():
    ops = workloads.qft_ops(range(12))
    kinds = [o.kind for o in ops]
    assert kinds.count("h") == 12 and kinds.count("p") == 66 and kinds.count("swap") == 6


@pytest.mark.parametrize("n", [2, 3, 6, 9])
def test_bell_and_ghz(n):
    st = oracle.OracleState(n)
    st.apply_matrix(oracle.GATES_1Q["h"], [0])
    for q in range(n - 1):
        st.apply_matrix(oracle.GATES_1Q["x"], [q + 1], [q])
    expect = np.zeros(1 << n, dtype=np.complex128)
    expect[0] = expect[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(st.psi, expect, atol=1e-15)


def test_norm_is_preserved_and_echo_returns_to_zero():
    circ = workloads.layered_circuit(8, seed=4, n_gates=120)
    st = oracle.run_circuit(circ)
    assert abs(st.norm2() - 1.0) < 1e-13
    # C then C^dagger returns |0...0>
    for op in reversed(circ.ops):
        U = oracle.gate_matrix(op.kind, op.params)
        st.apply_matrix(U.conj().T, op.targets, op.controls)
    e0 = np.zeros(1 << 8)
    e0[0] = 1
    np.testing.assert_allclose(st.psi, e0, atol=1e-12)


def test_add_qubits_appends_high_zero_qubits():
    psi = rand_state(3, 2)
    st = oracle.OracleState(3, psi=psi)
    assert st.add_qubits(2) == 3
    np.testing.assert_allclose(st.psi, np.kron(np.array([1, 0, 0, 0]), psi), atol=0)


# -- permutations -------------------------------------------------------------------

def test_mulmod_maps_basis_states_exactly():
    # register qubits 1..4 (qubit 1 = MSB), control qubit 0; x -> 7x mod 15
    reg = [1, 2, 3, 4]
    for x in range(16):
        for ctrl in (0, 1):
            i = ctrl
            for a, q in enumerate(reg):
                i |= ((x >> (3 - a)) & 1) << q
            psi = np.zeros(32, dtype=np.complex128)
            psi[i] = 1
            st = oracle.OracleState(5, psi=psi)
            st.apply_mulmod(7, 15, reg, [0])
            y = (7 * x) % 15 if (ctrl and x < 15) else x
            j = ctrl
            for a, q in enumerate(reg):
                j |= ((y >> (3 - a)) & 1) << q
            assert np.flatnonzero(st.psi).tolist() == [j]


def test_perm_table_and_bijectivity_check():
    n = 4
    f = [3, 0, 2, 1]
    psi = rand_state(n, 11)
    st = oracle.OracleState(n, psi=psi)
    st.apply_perm(f, [2, 0])  # register value = 2*bit2 + bit0
    for i in range(16):
        x = 2 * ((i >> 2) & 1) + (i & 1)
        y = f[x]
        j = (i & ~0b101) | ((y >> 1) << 2) | (y & 1)
        assert st.psi[j] == psi[i]
    with pytest.raises(ValueError):
        st.apply_perm([0, 0, 1, 2], [2, 0])
    with pytest.raises(ValueError):
        st.apply_mulmod(16, 15, [0, 1, 2, 3])  # c must be reduced mod N


def test_mulmod_non_coprime_rejected_as_non_bijective():
    st = oracle.OracleState(4)
    with pytest.raises(ValueError):
        st.apply_mulmod(5, 15, [0, 1, 2, 3])


# -- measurement ---------------------------------------------------------------------

def test_measurement_probability_collapse_and_rule():
    n = 5
    psi = rand_state(n, 21)
    for q in range(n):
        marg0 = float(np.sum(np.abs(psi.reshape(-1, 2, 1 << q)[:, 0, :]) ** 2))
        p0 = oracle.OracleState(n, psi=psi).prob0(q)
        assert abs(p0 - marg0) < 1e-14
        for u in (0.0, p0 - 1e-9, p0, 0.999):  # u == P0 exactly must give outcome 1
            st = oracle.OracleState(n, 1, psi=psi)
            m = st.measure([q], [u], [0])
            assert st.last_p0[0] == p0
            assert m == (0 if u < p0 else 1) and st.cbits[0] == m
            proj = kron_list({q: P1 if m else P0}, n)
            post = proj @ psi
            post /= np.linalg.norm(post)
            np.testing.assert_allclose(st.psi, post, atol=1e-14)


def test_measure_basis_states_is_deterministic():
    for bit in (0, 1):
        st = oracle.OracleState(2)
        if bit:
            st.apply_matrix(oracle.GATES_1Q["x"], [1])
        assert st.measure([1], [0.0]) == bit
        assert st.measure([1], [0.999999]) == bit


def test_multi_qubit_measure_register_value_and_joint_law():
    n = 3
    psi = rand_state(n, 8)
    st = oracle.OracleState(n, 3, psi=psi)
    v = st.measure([2, 0, 1], [0.3, 0.6, 0.1], [0, 1, 2])
    assert v == (st.cbits[0] << 2) | (st.cbits[1] << 1) | st.cbits[2]
    # P of the sampled branch equals product of the sequential conditionals
    idx = (st.cbits[0] << 2) | st.cbits[1] | (st.cbits[2] << 1)
    p = abs(psi[idx]) ** 2
    prod = 1.0
    for p0, m in zip(st.last_p0, st.cbits):
        prod *= p0 if m == 0 else 1 - p0
    assert abs(p - prod) < 1e-13
    assert abs(abs(st.psi[idx]) - 1) < 1e-13


def test_rphase_angles():
    st = oracle.OracleState(1, 2)
    st.apply_matrix(oracle.GATES_1Q["h"], [0])
    st.cbits[:] = [1, 0]
    st.rphase(0, [0])  # e = 1, m_1 = 1 -> theta = -pi/2 (S dagger)
    np.testing.assert_allclose(st.psi, np.array([1, -1j]) / math.sqrt(2), atol=1e-15)
    st2 = oracle.OracleState(1, 2)
    st2.apply_matrix(oracle.GATES_1Q["x"], [0])
    st2.cbits[:] = [1, 1]
    st2.rphase(0, [0, 1])  # theta = -2 pi (1/4 + 1/8)
    np.testing.assert_allclose(st2.psi, [0, np.exp(-1j * 3 * math.pi / 4)], atol=1e-15)


# -- Kitaev order finding -------------------------------------------------------------

def multiplicative_order(a, N):
    r, x = 1, a % N
    while x != 1:
        x = x * a % N
        r += 1
    return r


def qpe_closed_form(r, t):
    """P(y) = (1/r) sum_s |2^-t sum_{x<2^t} exp(2 pi i x (s/r - y/2^t))|^2."""
    T = 1 << t
    y = np.arange(T)
    P = np.zeros(T)
    for s in range(r):
        delta = s / r - y / T
        num = np.exp(2j * math.pi * delta * T) - 1
        den = np.exp(2j * math.pi * delta) - 1
        amp = np.where(np.abs(den) < 1e-12, T, num / np.where(np.abs(den) < 1e-12, 1, den)) / T
        P += np.abs(amp) ** 2 / r
    return P


def forced_uniforms(y, t):
    return [0.0 if ((y >> e) & 1) == 0 else 1.0 - 2.0 ** -53 for e in range(t)]


def test_kitaev_n15_printed_shape_and_peaks():
    g = load_golden("paper_values.txt")
    N, a = 15, g["default_base_a"]
    t = workloads.paper_stage_count(N)
    assert t == g["n15_cbits"]
    assert N.bit_length() == g["n15_work_qubits"]
    assert N.bit_length() + 2 * N.bit_length() == g["n15_3nx1_qubits"]
    # r = 4 divides 2^8, so y in {0, 64, 128, 192} each with probability 1/4
    for y in range(1 << t):
        expect = 0.25 if y in (0, 64, 128, 192) else 0.0
        if expect == 0.0:
            continue
        got, bits, probs, st = oracle.kitaev_order_finding(N, a, t, forced_uniforms(y, t))
        assert got == y
        assert abs(np.prod(probs) - expect) < 1e-12
        assert all(abs(p - 1) < 1e-12 for p in probs[:6])
    rng = workloads.SplitMix64(5)
    for _ in range(20):
        us = [rng.uniform() for _ in range(t)]
        y, *_ = oracle.kitaev_order_finding(N, a, t, us)
        assert y in (0, 64, 128, 192)


@pytest.mark.parametrize("N,a", [(21, 2), (35, 3), (33, 5)])
def test_kitaev_stage_product_equals_closed_form(N, a):
    b = N.bit_length()
    t = 2 * b
    r = multiplicative_order(a, N)
    P = qpe_closed_form(r, t)
    assert abs(P.sum() - 1) < 1e-9
    ys = np.argsort(P)[::-1][:12]
    for y in ys:
        if P[y] < 1e-6:
            continue
        got, bits, probs, st = oracle.kitaev_order_finding(N, a, t, forced_uniforms(int(y), t))
        assert got == y
        assert abs(np.prod(probs) - P[y]) < 1e-9
        assert abs(st.norm2() - 1) < 1e-12


def test_kitaev_samples_peak_at_multiples_of_2t_over_r():
    N, a = 21, 2
    t = 10
    r = multiplicative_order(a, N)  # 6
    rng = workloads.SplitMix64(77)
    hits = 0
    trials = 40
    for _ in range(trials):
        y, *_ = oracle.kitaev_order_finding(N, a, t, [rng.uniform() for _ in range(t)])
        frac = y * r / (1 << t)
        if abs(frac - round(frac)) < 0.5 * r / (1 << t) * 2:
            hits += 1
    # the closed form puts ~> 0.8 of the mass within one bin of a peak s 2^t / r
    assert hits >= 0.6 * trials


def test_paper_printed_order_values():
    g = load_golden("paper_values.txt")
    N = g["n13564597"]
    assert N.bit_length() + 1 == g["n13564597_nx2n_qubits"]
    assert g["n961307"].bit_length() + 1 == g["n961307_nx2n_qubits"]
    r = multiplicative_order(g["default_base_a"], N)
    assert r == g["n13564597_order"]
    assert r % g["n13564597_partial"] == 0 and r // g["n13564597_partial"] == 4


@pytest.mark.parametrize("N,a", [(15, 7), (21, 2), (35, 3)])
def test_kitaev_op_list_matches_the_stage_by_stage_oracle(N, a):
    """workloads.kitaev_circuit (the op list every Kitaev GPU test feeds to both
    sides) walked op by op reproduces oracle.kitaev_order_finding (the nx2n stages
    of Appendix A written against the oracle API, pinned above by the closed-form
    phase-estimation law): the same bits and the same final state."""
    t = 2 * N.bit_length()
    rng = workloads.SplitMix64(900 + N)
    u = [rng.uniform() for _ in range(t)]
    y, bits, _, st = oracle.kitaev_order_finding(N, a, t, u)
    circ = workloads.kitaev_circuit(N, a, uniforms=u)
    assert circ.n_cbits == t and circ.n_qubits == N.bit_length() + 1
    ref = oracle.run_circuit(circ)
    assert [int(x) for x in ref.cbits] == bits
    np.testing.assert_allclose(ref.psi, st.psi, atol=1e-13)


def test_all_core_oracle_build_is_bit_identical():
    """The OpenMP build of the oracle (used only to time it on every host core)
    splits the gate loop's independent groups across threads; each group's
    arithmetic is unchanged, so the states agree bit for bit."""
    circ = workloads.layered_circuit(14, seed=5, n_gates=90, qft=True)
    a = oracle.OracleState(14)
    b = oracle.OracleState(14, openmp=True)
    for op in circ.ops:
        a.apply_op(op)
        b.apply_op(op)
    assert np.array_equal(a.psi, b.psi)


# -- conventional order finding (the 3nx1 branch) ---------------------------------

def register_marginal(psi, qubits):
    """P(value) of a register (first-listed qubit = MSB) from a full state."""
    n = int(np.log2(psi.size))
    idx = np.arange(psi.size)
    val = np.zeros(psi.size, dtype=np.int64)
    for q in qubits:
        val = (val << 1) | ((idx >> q) & 1)
    return np.bincount(val, weights=np.abs(psi) ** 2, minlength=1 << len(qubits))


def shor_3nx1_amplitude(y, x0, r, t):
    """Control-register amplitude after the forward QFT when the control register
    holds the uniform superposition of x = x0, x0 + r, ... < 2^t (what measuring the
    work register leaves): (M 2^t)^-1/2 sum_{m<M} exp(2 pi i (x0 + m r) y / 2^t)."""
    T = 1 << t
    M = (T - x0 + r - 1) // r
    x = x0 + r * np.arange(M)
    return np.exp(2j * math.pi * np.outer(np.atleast_1d(y), x) / T).sum(axis=1) / math.sqrt(M * T)


def reg_value(bits):
    """Register value from measured bits, first bit the MSB."""
    v = 0
    for m in bits:
        v = 2 * v + int(m)
    return v


def ops_until_last_measure(circ):
    k = max(i for i, op in enumerate(circ.ops) if op.kind == "measure")
    return circ.ops[:k]


def test_3nx1_n15_exact_outcome_law():
    """N = 15, a = 2 (12 qubits: 8 control + 4 work, the paper's printed shape):
    before the work register is measured it holds 1, 2, 4, 8 with probability 1/4
    each; afterwards the QFT leaves the control register on y = 0, 64, 128, 192
    with probability 1/4 each (r = 4 divides 2^8) and nothing anywhere else."""
    g = load_golden("paper_values.txt")
    N, a = 15, g["default_base_a"]
    circ = workloads.shor_3nx1_circuit(N, a)
    assert circ.n_qubits == g["n15_3nx1_qubits"]
    t, b = workloads.paper_stage_count(N), N.bit_length()
    assert t == g["n15_cbits"]
    ctrl, work = list(range(t)), list(range(t, t + b))
    st = oracle.OracleState(circ.n_qubits, circ.n_cbits)
    for op in circ.ops:
        if op.kind == "measure" and tuple(op.targets) == tuple(work):
            Pw = register_marginal(st.psi, work)
            np.testing.assert_allclose(Pw[[1, 2, 4, 8]], 0.25, atol=1e-12)
            assert abs(Pw.sum() - 1) < 1e-12
        if op.kind == "measure" and tuple(op.targets) == tuple(ctrl):
            Py = register_marginal(st.psi, ctrl)
            expect = np.zeros(1 << t)
            expect[[0, 64, 128, 192]] = 0.25
            np.testing.assert_allclose(Py, expect, atol=1e-12)
        st.apply_op(op)
    w = reg_value(st.cbits[:b])
    y = reg_value(st.cbits[b:])
    assert w in (1, 2, 4, 8) and y in (0, 64, 128, 192)


@pytest.mark.parametrize("N,a", [(21, 2), (33, 5), (35, 3)])
def test_3nx1_state_equals_the_closed_form(N, a):
    """General N (r need not divide 2^t): after the work register is measured at
    w = a^x0 mod N and the QFT sequence has run, every amplitude of the state equals
    the closed form on work value w and is zero elsewhere; averaged over x0, the
    control-register law is the phase-estimation closed form that pins the Kitaev
    run above."""
    circ = workloads.shor_3nx1_circuit(N, a, seed=11)
    t, b = workloads.paper_stage_count(N), N.bit_length()
    st = oracle.OracleState(circ.n_qubits, circ.n_cbits)
    for op in ops_until_last_measure(circ):
        st.apply_op(op)
    r = multiplicative_order(a, N)
    w = reg_value(st.cbits[:b])
    x0 = next(x for x in range(r) if pow(a, x, N) == w)
    ys = np.arange(1 << t)
    A = shor_3nx1_amplitude(ys, x0, r, t)
    # index = sum_q bit_q 2^q with control qubit q = bit t-1-q of y, work qubit t+k = bit b-1-k of w
    yidx = np.zeros(1 << t, dtype=np.int64)
    for q in range(t):
        yidx |= ((ys >> (t - 1 - q)) & 1) << q
    widx = sum(((w >> (b - 1 - k)) & 1) << (t + k) for k in range(b))
    np.testing.assert_allclose(st.psi[yidx + widx], A, atol=1e-12)
    assert abs(np.sum(np.abs(st.psi[yidx + widx]) ** 2) - 1) < 1e-12
    # the x0-average of |A|^2 weighted by P(w) = M / 2^t is the Kitaev closed form
    T = 1 << t
    Py = sum(((T - x + r - 1) // r) / T * np.abs(shor_3nx1_amplitude(ys, x, r, t)) ** 2 for x in range(r))
    np.testing.assert_allclose(Py, qpe_closed_form(r, t), atol=1e-12)
