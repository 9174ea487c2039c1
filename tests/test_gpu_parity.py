"""GPU parity: libqk (through the C ABI) against the CPU oracle, element by element.

Tolerances: complex64 max |delta a| <= 1e-4 absolute and total-variation
distance <= 1e-5 on the output distribution, complex128 <= 1e-12; permutations,
measured bits and cbits bit-exact (a measured bit may differ only where the
uniform lies within the precision's bound of P0, which the helper reports).
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-4, "c128": 1e-12}
TV_TOL = {"c64": 1e-5, "c128": 1e-12}
MARGIN = {"c64": 1e-6, "c128": 1e-12}
MODES = ("plain", "fused")


@pytest.fixture(scope="module")
def qk():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07187_gb300 import qk as mod

    return mod


def tv(a, b):
    return 0.5 * float(np.sum(np.abs(np.abs(a) ** 2 - np.abs(b) ** 2)))


def check_state(got, ref, prec):
    err = float(np.max(np.abs(got.astype(np.complex128) - ref)))
    assert err <= TOL[prec], f"max |delta a| = {err:.3e}"
    assert tv(got.astype(np.complex128), ref) <= TV_TOL[prec]


def haar(d, rng):
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / math.sqrt(2)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def new_ctx(qk, n, prec, mode, psi=None, ncb=0, **kw):
    ctx = qk.Context(prec, mode, **kw)
    ctx.add_qubits(n)
    if ncb:
        ctx.add_cbits(ncb)
    if psi is not None:
        ctx.set_state(psi)
    return ctx


# -- single gates on random states ---------------------------------------------

@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [1, 2, 5, 11, 15])
def test_one_qubit_gates_every_target(qk, prec, mode, n):
    rng = np.random.default_rng(n)
    psi = workloads.random_state(n, 40 + n)
    ctx = new_ctx(qk, n, prec, mode, psi)
    ref = oracle.OracleState(n, psi=psi)
    for q in range(n):
        th, ph, la = rng.uniform(0, 2 * math.pi, 3)
        ctx.apply_gate("u3", [q], params=[th, ph, la])
        ref.apply_matrix(oracle.u3(th, ph, la), [q])
        g = ["h", "x", "y", "z", "s", "t", "sdg"][q % 7]
        ctx.apply_gate(g, [q])
        ref.apply_matrix(oracle.GATES_1Q[g], [q])
    check_state(ctx.get_state(), ref.psi, prec)
    ctx.close()


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("target,controls", [(0, [1]), (3, [0]), (1, [0, 4]), (7, [2, 5, 0]), (12, [13]),
                                             (5, [12, 1])])
def test_controlled_gates(qk, prec, mode, target, controls):
    n = 14
    rng = np.random.default_rng(target * 17 + len(controls))
    psi = workloads.random_state(n, 7)
    U = haar(2, rng)
    gid_ctx = new_ctx(qk, n, prec, mode, psi)
    gid = gid_ctx.define_gate_matrix(U)
    gid_ctx.apply_gate(gid, [target], controls)
    gid_ctx.apply_gate("p", [target], controls, params=[0.37])
    gid_ctx.apply_gate("x", [target], controls)
    ref = oracle.OracleState(n, psi=psi)
    ref.apply_matrix(U, [target], controls)
    ref.apply_matrix(oracle.phase(0.37), [target], controls)
    ref.apply_matrix(oracle.GATES_1Q["x"], [target], controls)
    check_state(gid_ctx.get_state(), ref.psi, prec)
    gid_ctx.close()


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("targets,controls", [((0, 1), ()), ((1, 0), ()), ((5, 2), (0,)), ((3, 9, 0), ()),
                                              ((2, 7, 4, 11), (1,)), ((0, 1, 2, 3, 4), ()),
                                              ((6, 1, 8, 3, 10, 0), ())])
def test_k_qubit_matrix_gates(qk, prec, targets, controls):
    n = 12
    rng = np.random.default_rng(len(targets) * 5 + sum(targets))
    U = haar(1 << len(targets), rng)
    psi = workloads.random_state(n, 8)
    ctx = new_ctx(qk, n, prec, "fused", psi)
    gid = ctx.define_gate_matrix(U)
    ctx.apply_gate(gid, targets, controls)
    ref = oracle.OracleState(n, psi=psi)
    ref.apply_matrix(U, targets, controls)
    check_state(ctx.get_state(), ref.psi, prec)
    ctx.close()


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_diagonal_k_qubit_gate_and_swap_relabel(qk, prec):
    n = 9
    psi = workloads.random_state(n, 12)
    D = np.diag(np.exp(1j * np.array([0.0, 0.3, 0.0, -1.2])))
    ctx = new_ctx(qk, n, prec, "fused", psi)
    gid = ctx.define_gate_matrix(D)
    ctx.apply_gate(gid, [4, 1])
    ctx.apply_gate("swap", [0, 8])
    ctx.apply_gate("h", [0])
    ctx.apply_gate("swap", [3, 0])
    ctx.apply_gate("swap", [2, 6], controls=[5])
    ctx.apply_gate("x", [8], controls=[3])
    ref = oracle.OracleState(n, psi=psi)
    ref.apply_matrix(D, [4, 1])
    ref.apply_matrix(oracle.SWAP, [0, 8])
    ref.apply_matrix(oracle.GATES_1Q["h"], [0])
    ref.apply_matrix(oracle.SWAP, [3, 0])
    ref.apply_matrix(oracle.SWAP, [2, 6], [5])
    ref.apply_matrix(oracle.GATES_1Q["x"], [8], [3])
    check_state(ctx.get_state(), ref.psi, prec)
    ctx.close()


# -- permutations --------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_mulmod_permutation_bit_exact(qk, prec):
    n = 13
    N, c = 187, 23  # 8-bit register, gcd(23, 187) = 1
    reg = [9, 2, 4, 11, 1, 7, 12, 5]
    psi = workloads.random_state(n, 14)
    ctx = new_ctx(qk, n, prec, "fused", psi)
    gid = ctx.define_gate_perm_mulmod(8, c, N)
    ctx.apply_gate(gid, reg, [3])
    got = ctx.get_state()
    ref = oracle.OracleState(n, psi=psi.astype(np.complex64 if prec == "c64" else np.complex128))
    ref.apply_mulmod(c, N, reg, [3])
    # a permutation moves amplitudes without arithmetic: bit-exact
    assert np.array_equal(got, ref.psi.astype(got.dtype))
    ctx.close()


@pytest.mark.parametrize("reg", [list(range(4, 12)), list(range(11, 3, -1)), [0, 1, 2, 3, 4, 5, 6, 7]])
def test_mulmod_on_contiguous_registers_bit_exact(qk, reg):
    # registers on consecutive physical bits take the bit-field index path
    # (first-listed qubit lowest: bit-reversed field; highest: the field itself)
    n = 13
    N, c = 211, 37
    psi = workloads.random_state(n, 16)
    ctx = new_ctx(qk, n, "c64", "fused", psi)
    gid = ctx.define_gate_perm_mulmod(8, c, N)
    ctrl = 12 if 12 not in reg else 3
    ctx.apply_gate(gid, reg, [ctrl])
    ref = oracle.OracleState(n, psi=psi.astype(np.complex64))
    ref.apply_mulmod(c, N, reg, [ctrl])
    assert np.array_equal(ctx.get_state(), ref.psi)
    f = np.random.default_rng(4).permutation(256).astype(np.uint64)
    tid = ctx.define_gate_perm_table(f)
    ctx.apply_gate(tid, reg)
    ref.apply_perm(f, reg)
    assert np.array_equal(ctx.get_state(), ref.psi)
    ctx.close()


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("reg,ctrls", [
    ([9, 2, 4, 11, 1, 7, 12, 5], [3, 0, 6, 10, 8]),                  # scattered register and controls
    (list(range(6, 14)), [5, 4, 3, 2, 1, 0, 14, 15, 16, 17]),       # contiguous register, 10 controls (2 groups)
])
def test_modexp_equals_controlled_mulmods_bit_exact(qk, prec, reg, ctrls):
    """One modular-exponentiation call against the oracle's controlled
    multiplications applied one after another (Appendix A, 3nx1 branch): a
    permutation, so bit-exact; the qubit map is relabelled first (SWAPs) so that
    the call's logical qubits sit elsewhere physically."""
    n = 18
    N, a = 221, 7                      # 221 = 13 * 17, gcd(7, 221) = 1
    mults = [pow(a, 1 << j, N) for j in range(len(ctrls))]
    psi = workloads.random_state(n, 31)
    ctx = new_ctx(qk, n, prec, "fused", psi)
    ctx.apply_gate("swap", [0, 13])
    ctx.apply_gate("swap", [5, 17])
    ctx.apply_modexp(reg, ctrls, mults, N)
    got = ctx.get_state()
    ref = oracle.OracleState(n, psi=psi.astype(np.complex64 if prec == "c64" else np.complex128))
    ref.apply_matrix(oracle.gate_matrix("swap"), [0, 13])
    ref.apply_matrix(oracle.gate_matrix("swap"), [5, 17])
    for c, m in zip(ctrls, mults):
        ref.apply_mulmod(m, N, reg, [c])
    assert np.array_equal(got, ref.psi.astype(got.dtype))
    ctx.close()


def test_modexp_condition_and_rejections(qk):
    n = 14
    psi = workloads.random_state(n, 33)
    ctx = new_ctx(qk, n, "c64", "plain", psi, ncb=2)
    reg, ctrls = [4, 5, 6, 7, 8, 9, 10, 11], [0, 1, 2]
    ctx.apply_modexp(reg, ctrls, [2, 4, 16], 255, cond=[1])          # cbit 1 is 0: nothing happens
    assert np.array_equal(ctx.get_state(), psi.astype(np.complex64))
    for args, status in [((reg, ctrls, [3, 4, 16], 255), "QK_ENOTBIJECTIVE"),   # gcd(3, 255) = 3
                         ((reg, ctrls, [2, 4, 300], 255), "QK_EINVAL"),          # multiplier >= N
                         ((reg, [0, 4, 2], [2, 4, 16], 255), "QK_EINVAL"),       # control among the targets
                         ((reg, ctrls, [2, 4, 16], 257), "QK_EINVAL"),           # N > 2^8
                         ((reg, [0, 1, 1], [2, 4, 16], 255), "QK_EINVAL")]:      # repeated control
        with pytest.raises(qk.QKError, match=status):
            ctx.apply_modexp(*args)
    assert np.array_equal(ctx.get_state(), psi.astype(np.complex64))
    ctx.close()


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n", [1, 3, 6, 11, 15])
def test_qubit_map_undone_bit_exact(qk, prec, n):
    """SWAPs only edit the logical -> physical qubit map; reading the state back
    undoes the map with one tiled gather (tiles over the low five bits on both
    sides).  A random chain of SWAPs against the oracle's SWAP gates: bit-exact."""
    rng = np.random.default_rng(100 + n)
    psi = workloads.random_state(n, 40 + n)
    ctx = new_ctx(qk, n, prec, "fused", psi)
    ref = oracle.OracleState(n, psi=psi.astype(np.complex64 if prec == "c64" else np.complex128))
    for _ in range(3 * n):
        if n < 2:
            break
        a, b = (int(x) for x in rng.choice(n, size=2, replace=False))
        ctx.apply_gate("swap", [a, b])
        ref.apply_matrix(oracle.gate_matrix("swap"), [a, b])
    got = ctx.get_state()
    assert np.array_equal(got, ref.psi.astype(got.dtype))
    ctx.close()


def test_perm_table_and_rejections(qk):
    n = 6
    rng = np.random.default_rng(3)
    f = rng.permutation(16).astype(np.uint64)
    psi = workloads.random_state(n, 15)
    ctx = new_ctx(qk, n, "c128", "fused", psi)
    gid = ctx.define_gate_perm_table(f)
    ctx.apply_gate(gid, [5, 0, 3, 2])
    ref = oracle.OracleState(n, psi=psi)
    ref.apply_perm(f, [5, 0, 3, 2])
    assert np.array_equal(ctx.get_state(), ref.psi)
    with pytest.raises(qk.QKError) as e:
        ctx.define_gate_perm_table([0, 0, 1, 2])
    assert e.value.status == qk.QK_ENOTBIJECTIVE
    with pytest.raises(qk.QKError) as e:
        ctx.define_gate_perm_mulmod(4, 5, 15)
    assert e.value.status == qk.QK_ENOTBIJECTIVE
    with pytest.raises(qk.QKError) as e:
        ctx.apply_gate("h", [6])
    assert e.value.status == qk.QK_EINVAL
    with pytest.raises(qk.QKError):
        ctx.define_gate_matrix(np.array([[1, 1], [0, 1]]))
    ctx.close()


# -- measurement and classical control ---------------------------------------------------

@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("mode", MODES)
def test_measurement_bits_and_collapse(qk, prec, mode):
    n = 12
    psi = workloads.random_state(n, 16)
    rng = workloads.SplitMix64(99)
    qubits = [0, 5, 11, 3, 7]
    us = [rng.uniform() for _ in qubits]
    ctx = new_ctx(qk, n, prec, mode, psi, ncb=len(qubits))
    v = ctx.measure(qubits, us, list(range(len(qubits))))
    ref = oracle.OracleState(n, len(qubits), psi=psi)
    rv = ref.measure(qubits, us, list(range(len(qubits))))
    margins = [abs(u - p) for u, p in zip(us, ref.last_p0)]
    if min(margins) > MARGIN[prec]:
        assert v == rv
        assert list(ctx.read_cbits()) == list(ref.cbits)
        check_state(ctx.get_state(), ref.psi, prec)
    ctx.close()


@pytest.mark.parametrize("mode", MODES)
def test_classical_condition_and_rphase(qk, mode):
    n = 7
    psi = workloads.random_state(n, 17)
    ctx = new_ctx(qk, n, "c128", mode, psi, ncb=4)
    ref = oracle.OracleState(n, 4, psi=psi)
    ctx.write_cbits(0, [1, 0, 1, 1])
    ref.cbits[:] = [1, 0, 1, 1]
    ctx.apply_gate("x", [2], cond=[0])          # acts
    ctx.apply_gate("h", [4], cond=[0, 1])       # does not act
    ctx.apply_gate("u3", [6], controls=[1], cond=[2, 3], params=[0.3, 0.2, 0.1])
    ctx.apply_rphase_cbits(0, [0, 1, 2, 3])
    ctx.apply_rphase_cbits(5, [3])
    ref.apply_matrix(oracle.GATES_1Q["x"], [2])
    ref.apply_matrix(oracle.u3(0.3, 0.2, 0.1), [6], [1])
    ref.rphase(0, [0, 1, 2, 3])
    ref.rphase(5, [3])
    check_state(ctx.get_state(), ref.psi, "c128")
    ctx.close()


# -- whole workloads --------------------------------------------------------------------------

def test_plain_c128_12q_circuit(qk):
    circ = workloads.plain_c128_circuit(seed=1)
    ref = oracle.run_circuit(circ)
    for mode in MODES:
        ctx = qk.run_circuit(circ, "c128", mode)
        bits = ctx.read_cbits()
        got = ctx.get_state()
        assert list(bits) == list(ref.cbits)
        check_state(got, ref.psi, "c128")
        ctx.close()


@pytest.mark.parametrize("n", [10, 14, 17])
@pytest.mark.parametrize("mode", MODES)
def test_layered_circuit_c64(qk, n, mode):
    circ = workloads.layered_circuit(n, seed=2, n_gates=500)
    ref = oracle.run_circuit(circ)
    ctx = qk.run_circuit(circ, "c64", mode)
    check_state(ctx.get_state(), ref.psi, "c64")
    ctx.close()


@pytest.mark.parametrize("b", [4, 6, 12])
def test_kitaev_order_finding_bits_exact(qk, b):
    N, a = (15, 7) if b == 4 else workloads.kitaev_parameters(b, seed=3)
    circ = workloads.kitaev_circuit(N, a, seed=5)
    ref = oracle.run_circuit(circ)
    for mode in MODES:
        ctx = qk.run_circuit(circ, "c64", mode)
        assert list(ctx.read_cbits()) == [int(x) for x in ref.cbits], mode
        check_state(ctx.get_state(), ref.psi, "c64")
        ctx.close()


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_order_finding_to_factors_n15(qk, seed):
    # the whole pipeline: fused Kitaev stages on the GPU, then continued fractions
    # and gcds on the host; for a = 7 the phases are s/4 exactly (r = 4 divides 2^8)
    from paper_1908_07187_gb300 import shor

    circ = workloads.kitaev_circuit(15, 7, seed=seed)
    ref = oracle.run_circuit(circ)
    ctx = qk.Context("c64", "fused")
    ctx.add_qubits(circ.n_qubits)
    ctx.add_cbits(circ.n_cbits)
    qk.run_kitaev_fused(ctx, circ)
    bits = [int(x) for x in ctx.read_cbits()]
    ctx.close()
    assert bits == [int(x) for x in ref.cbits]
    y = shor.outcome_from_bits(bits)
    assert y % 64 == 0
    r = shor.order_from_outcome(y, circ.n_cbits, 7, 15)
    if y:
        assert r == 4
        assert shor.factors_from_order(7, r, 15) == (3, 5)
    else:
        assert r is None


def oracle_with_margin(circ):
    """The oracle's run of a circuit and the smallest |u - P0| over its measured
    qubits (a bit may legitimately differ only where that is below the precision's
    bound)."""
    ref = oracle.OracleState(circ.n_qubits, circ.n_cbits)
    margin = 1.0
    for op in circ.ops:
        ref.apply_op(op)
        if op.kind == "measure":
            margin = min([margin] + [abs(u - p0) for u, p0 in zip(op.uniforms, ref.last_p0)])
    return ref, margin


@pytest.mark.parametrize("N,a", [(15, 2), (15, 7), (21, 2), (33, 5), (35, 3)])
@pytest.mark.parametrize("prec,mode", [("c64", "plain"), ("c64", "fused"), ("c128", "plain")])
def test_shor_3nx1_against_oracle(qk, N, a, prec, mode):
    """The conventional (3nx1) order-finding circuit of Appendix A: 2b+1 or 2b
    control qubits, b work qubits, controlled mul-mod gathers, the work register
    measured mid-circuit, the QFT sequence, the control register measured: cbits
    bit-exact and the final state element by element."""
    circ = workloads.shor_3nx1_circuit(N, a, seed=7)
    ref, margin = oracle_with_margin(circ)
    assert margin > MARGIN[prec]
    ctx = qk.run_circuit(circ, prec, mode)
    assert list(ctx.read_cbits()) == [int(x) for x in ref.cbits]
    check_state(ctx.get_state(), ref.psi, prec)
    ctx.close()


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_shor_3nx1_n21_to_factors(qk, seed):
    # the whole conventional pipeline: the GPU run, then continued fractions on the
    # control register's value (r = 6 for a = 2, which does not divide 2^9)
    from paper_1908_07187_gb300 import shor

    N, a = 21, 2
    circ = workloads.shor_3nx1_circuit(N, a, seed=seed)
    ref, margin = oracle_with_margin(circ)
    ctx = qk.run_circuit(circ, "c64", "fused")
    bits = [int(x) for x in ctx.read_cbits()]
    ctx.close()
    assert margin > MARGIN["c64"] and bits == [int(x) for x in ref.cbits]
    b, t = N.bit_length(), circ.n_cbits - N.bit_length()
    assert shor.register_from_bits(bits[:b]) in {pow(a, x, N) for x in range(6)}
    y = shor.register_from_bits(bits[b:])
    r = shor.order_from_outcome(y, t, a, N)
    if r is not None:
        assert r == 6 and shor.factors_from_order(a, r, N) in ((3, 7), (7, 3))


def test_add_qubits_keeps_state_and_counters(qk):
    psi = workloads.random_state(5, 19)
    ctx = new_ctx(qk, 5, "c64", "plain", psi)
    ctx.reset_counters()
    ctx.apply_gate("h", [2])
    assert ctx.counters()["launches"] == 1
    ctx.add_qubits(3)
    ref = oracle.OracleState(5, psi=psi)
    ref.apply_matrix(oracle.GATES_1Q["h"], [2])
    ref.add_qubits(3)
    check_state(ctx.get_state(), ref.psi, "c64")
    ctx.close()


# -- fused tile passes on random mixed circuits ------------------------------------------------

def random_mixed_ops(n, n_ops, seed, ncb=0):
    """Seeded random mix of 1-qubit gates with 0..2 controls, diagonal gates with
    controls, SWAPs and classically conditioned gates."""
    rng = np.random.default_rng(seed)
    ops = []
    kinds = ["u3", "h", "x", "y", "z", "s", "t", "p", "rz", "swap", "sdg"]
    for _ in range(n_ops):
        k = kinds[rng.integers(len(kinds))]
        qs = [int(x) for x in rng.choice(n, size=4, replace=False)]
        nc = int(rng.integers(0, 3))
        cond = ()
        if ncb and rng.random() < 0.15:
            cond = (int(rng.integers(ncb)),)
        if k == "swap":
            ops.append(workloads.Op("swap", (qs[0], qs[1]), controls=tuple(qs[2:2 + (nc > 1)]), cond=cond))
            continue
        params = ()
        if k == "u3":
            params = tuple(float(x) for x in rng.uniform(0, 2 * math.pi, 3))
        elif k in ("p", "rz"):
            params = (float(rng.uniform(0, 2 * math.pi)),)
        ops.append(workloads.Op(k, (qs[0],), controls=tuple(qs[1:1 + nc]), params=params, cond=cond))
    return ops


def oracle_apply(st, op):
    if op.cond and not all(st.cbits[c] for c in op.cond):
        return
    st.apply_matrix(oracle.gate_matrix(op.kind, op.params), op.targets, op.controls)


@pytest.mark.parametrize("n,seed", [(13, 1), (14, 2), (15, 3), (16, 4), (18, 5), (20, 6)])
def test_fused_random_mixed_circuits(qk, n, seed):
    ops = random_mixed_ops(n, 300, seed, ncb=3)
    psi = workloads.random_state(n, 60 + seed)
    ctx = new_ctx(qk, n, "c64", "fused", psi, ncb=3)
    ctx.write_cbits(0, [1, 0, 1])
    ref = oracle.OracleState(n, 3, psi=psi)
    ref.cbits[:] = [1, 0, 1]
    qk.run_ops(ctx, ops)
    for op in ops:
        oracle_apply(ref, op)
    check_state(ctx.get_state(), ref.psi, "c64")
    ctx.close()


@pytest.mark.parametrize("n", [13, 16, 19])
def test_fused_matches_plain_and_uses_few_passes(qk, n):
    circ = workloads.layered_circuit(n, seed=9, n_gates=400)
    got = {}
    for mode in MODES:
        ctx = qk.run_circuit(circ, "c64", mode)
        ctx.sync()
        got[mode] = (ctx.get_state(), ctx.counters())
        ctx.close()
    assert np.max(np.abs(got["fused"][0] - got["plain"][0])) < 1e-4
    assert got["fused"][1]["launches"] < got["plain"][1]["launches"] / 10


@pytest.mark.parametrize("targets", [(5, 6), (0, 9), (2, 13), (14, 3), (11, 12)])
def test_fused_two_qubit_diagonals_every_pattern(qk, targets):
    """Diagonal 2-qubit gates whose non-unit entries sit on the (0,0), (0,1),
    (1,0) and (1,1) patterns, between non-diagonal gates on the same qubits."""
    n = 15
    psi = workloads.random_state(n, 77 + sum(targets))
    ctx = new_ctx(qk, n, "c64", "fused", psi)
    ref = oracle.OracleState(n, psi=psi)
    diags = [np.diag(np.exp(1j * np.array(a))) for a in ([0.7, 0, 0, -1.1], [0, 0.4, 1.3, 0], [0, 2.0, 0, 0],
                                                         [0, 0, -0.6, 0], [math.pi, 0, 0, 0])]
    for D in diags:
        gid = ctx.define_gate_matrix(D)
        ctx.apply_gate(gid, targets)
        ref.apply_matrix(D, targets)
        ctx.apply_gate("h", [targets[0]])
        ref.apply_matrix(oracle.GATES_1Q["h"], [targets[0]])
        ctx.apply_gate("u3", [targets[1]], params=[0.3, 0.9, 1.7])
        ref.apply_matrix(oracle.u3(0.3, 0.9, 1.7), [targets[1]])
    check_state(ctx.get_state(), ref.psi, "c64")
    ctx.close()


@pytest.mark.parametrize("b", [16, 18, 20])
def test_kitaev_large_registers_bits_exact_against_oracle(qk, b):
    """Order finding at the b = 16..20-bit sizes of the benchmark configuration
    (17..21 qubits; the Abstract's 21-qubit run is the b = 20 shape): the fused
    stage calls and their CUDA-graph replay give the oracle's measured bits
    exactly and its final state within the complex64 bound."""
    N, a = workloads.kitaev_parameters(b, seed=3)
    circ = workloads.kitaev_circuit(N, a, seed=5)
    ref = oracle.run_circuit(circ)
    ctx = qk.Context("c64", "fused")
    ctx.add_qubits(circ.n_qubits)
    ctx.add_cbits(circ.n_cbits)
    qk.run_kitaev_fused(ctx, circ)
    assert list(ctx.read_cbits()) == [int(x) for x in ref.cbits]
    check_state(ctx.get_state(), ref.psi, "c64")
    ctx.sync()
    ctx.capture_begin()
    ctx.reset()
    qk.run_kitaev_fused(ctx, circ)
    g = ctx.capture_end()
    ctx.write_cbits(0, [0] * circ.n_cbits)
    g.launch()
    assert list(ctx.read_cbits()) == [int(x) for x in ref.cbits]
    check_state(ctx.get_state(), ref.psi, "c64")
    g.close()
    ctx.close()


@pytest.mark.parametrize("qubits", [[0], [7], [21], [3, 17]])
def test_measurement_probability_within_1e9_of_oracle(qk, qubits):
    """The complex64 measurement sums (compensated FP32 per thread, FP64 across)
    against the oracle's FP64 sums on the same complex64 amplitudes: a uniform
    1e-9 below the oracle's P0 reads 0 and 1e-9 above reads 1, for every decision
    of a sequential measurement, on a 22-qubit state whose P0 values sit near 1/2."""
    n = 22
    psi = workloads.random_state(n, 404).astype(np.complex64)
    ref = oracle.OracleState(n, psi=psi.astype(np.complex128))
    # the oracle's P0 of each decision in turn, each taken on the collapsed state
    base_u = [0.3] * len(qubits)
    probe = oracle.OracleState(n, psi=psi.astype(np.complex128))
    p0s = []
    for j, q in enumerate(qubits):
        p0s.append(probe.prob0(q))
        probe.measure([q], [base_u[j]])
    assert all(abs(p - 0.5) < 0.01 for p in p0s)
    for j in range(len(qubits)):
        for delta, want in ((-1e-9, 0), (1e-9, 1)):
            us = list(base_u)
            us[j] = p0s[j] + delta
            ctx = new_ctx(qk, n, "c64", "plain", psi)
            v = ctx.measure(qubits, us)
            bit = (v >> (len(qubits) - 1 - j)) & 1
            assert bit == want, (qubits, j, delta, p0s[j])
            ctx.close()
    _ = ref


@pytest.mark.parametrize("b,prec", [(4, "c64"), (6, "c128"), (12, "c64"), (14, "c64")])
def test_fused_kitaev_stage_matches_oracle_and_generic(qk, b, prec):
    N, a = (15, 7) if b == 4 else workloads.kitaev_parameters(b, seed=3)
    circ = workloads.kitaev_circuit(N, a, seed=21)
    ref = oracle.run_circuit(circ)
    ctx = qk.Context(prec, "fused")
    ctx.add_qubits(circ.n_qubits)
    ctx.add_cbits(circ.n_cbits)
    qk.run_kitaev_fused(ctx, circ)
    assert list(ctx.read_cbits()) == [int(x) for x in ref.cbits]
    check_state(ctx.get_state(), ref.psi, prec)
    gen = qk.run_circuit(circ, prec, "fused")
    np.testing.assert_allclose(ctx.get_state(), gen.get_state(), atol=TOL[prec])
    ctx.close()
    gen.close()


def test_fused_kitaev_stage_rejects_bad_arguments(qk):
    ctx = qk.Context("c64", "fused")
    ctx.add_qubits(5)
    ctx.add_cbits(2)
    gid = ctx.define_gate_perm_mulmod(4, 7, 15)
    u = ctx.define_gate_matrix(np.eye(2))
    with pytest.raises(qk.QKError):
        ctx.apply_kitaev_stage(0, u, [1, 2, 3, 4], [], 0.5, 0)        # not a permutation gate
    with pytest.raises(qk.QKError):
        ctx.apply_kitaev_stage(1, gid, [1, 2, 3, 4], [], 0.5, 0)      # control among the targets
    with pytest.raises(qk.QKError):
        ctx.apply_kitaev_stage(0, gid, [1, 2, 3, 4], [5], 0.5, 0)     # cbit out of range
    with pytest.raises(qk.QKError):
        ctx.apply_kitaev_stage(0, gid, [1, 2, 3, 4], [], 1.0, 0)      # uniform outside [0, 1)
    ctx.close()


# -- CUDA graph capture ------------------------------------------------------------------------

def test_graph_replay_of_a_kitaev_run_matches_direct_run(qk):
    N, a = workloads.kitaev_parameters(8, seed=3)
    circ = workloads.kitaev_circuit(N, a, seed=9)
    ref = oracle.run_circuit(circ)
    ctx = qk.Context("c64", "fused")
    ctx.add_qubits(circ.n_qubits)
    ctx.add_cbits(circ.n_cbits)
    qk.run_kitaev_fused(ctx, circ)          # defines the gates, allocates the gather buffer
    ctx.sync()
    ctx.capture_begin()
    with pytest.raises(qk.QKError) as e:
        ctx.read_cbits()
    assert e.value.status == qk.QK_ESTATE
    ctx.reset()
    qk.run_kitaev_fused(ctx, circ)
    g = ctx.capture_end()
    for _ in range(3):
        ctx.write_cbits(0, [0] * circ.n_cbits)
        g.launch()
        assert list(ctx.read_cbits()) == [int(x) for x in ref.cbits]
        check_state(ctx.get_state(), ref.psi, "c64")
    g.close()
    ctx.close()


def test_graph_replays_compose_with_relabels_and_odd_gathers(qk):
    n = 14
    psi = workloads.random_state(n, 5)
    ctx = new_ctx(qk, n, "c64", "fused", psi)
    gid = ctx.define_gate_perm_mulmod(5, 7, 29)
    ctx.apply_gate(gid, [9, 3, 12, 0, 6], [1])   # allocates the gather buffer once
    ref = oracle.OracleState(n, psi=psi)
    ref.apply_mulmod(7, 29, [9, 3, 12, 0, 6], [1])
    ctx.capture_begin()
    ctx.apply_gate("h", [0])
    ctx.apply_gate("swap", [0, 11])
    ctx.apply_gate("u3", [11], params=[0.4, 1.0, 2.0])
    ctx.apply_gate(gid, [9, 3, 12, 0, 6], [1])   # one out-of-place gather: odd
    ctx.apply_gate("p", [4], controls=[13], params=[0.9])
    g = ctx.capture_end()
    for _ in range(2):
        g.launch()
        ref.apply_matrix(oracle.GATES_1Q["h"], [0])
        ref.apply_matrix(oracle.SWAP, [0, 11])
        ref.apply_matrix(oracle.u3(0.4, 1.0, 2.0), [11])
        ref.apply_mulmod(7, 29, [9, 3, 12, 0, 6], [1])
        ref.apply_matrix(oracle.phase(0.9), [4], [13])
    check_state(ctx.get_state(), ref.psi, "c64")
    g.close()
    ctx.close()
