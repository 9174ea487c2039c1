"""Dense 5-qubit blocks on the tensor cores (3xTF32 tcgen05 GEMM) against the
oracle and against the CUDA-core path, on whole tiles and ragged tails."""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qk():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07187_gb300 import qk as mod

    return mod


def haar(d, rng):
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / math.sqrt(2)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


@pytest.mark.parametrize("n,targets", [(12, (4, 3, 2, 1, 0)), (5, (4, 3, 2, 1, 0)), (10, (0, 1, 2, 3, 4)),
                                       (14, (2, 0, 4, 1, 3)), (20, (3, 4, 0, 2, 1))])
def test_block_tc_matches_oracle(qk, n, targets):
    rng = np.random.default_rng(n + sum(t * 7 ** i for i, t in enumerate(targets)))
    U = haar(32, rng)
    psi = workloads.random_state(n, 300 + n)
    ctx = qk.Context("c64", "plain")
    ctx.add_qubits(n)
    ctx.set_state(psi)
    gid = ctx.define_gate_matrix(U)
    ctx.apply_gate(gid, targets)
    ctx.apply_gate(gid, targets)            # twice: the cached split matrices are reused
    ctx.sync()
    assert ctx.counters()["launches"] >= 2
    got = ctx.get_state().astype(np.complex128)
    ref = oracle.OracleState(n, psi=psi)
    ref.apply_matrix(U, list(targets))
    ref.apply_matrix(U, list(targets))
    err = float(np.max(np.abs(got - ref.psi)))
    assert err <= 1e-5, err
    ctx.close()


def test_block_tc_agrees_with_cuda_core_path(qk):
    n = 16
    rng = np.random.default_rng(11)
    U = haar(32, rng)
    psi = workloads.random_state(n, 12)
    out = []
    for tc in (True, False):
        ctx = qk.Context("c64", "fused", tensor_cores=tc)
        ctx.add_qubits(n)
        ctx.set_state(psi)
        gid = ctx.define_gate_matrix(U)
        ctx.apply_gate("h", [7])
        ctx.apply_gate(gid, [1, 0, 3, 2, 4])
        ctx.apply_gate("x", [2], controls=[9])
        out.append(ctx.get_state())
        ctx.close()
    assert np.max(np.abs(out[0] - out[1])) < 1e-5


@pytest.mark.parametrize("n,blocks", [(14, [(9, 12, 5, 13, 7)]), (16, [(4, 3, 2, 1, 0), (15, 11, 8, 6, 10)]),
                                      (20, [(19, 18, 17, 16, 15), (2, 9, 14, 0, 6), (4, 3, 2, 1, 0)])])
def test_block_tc_on_any_qubits_matches_oracle(qk, n, blocks):
    """5-qubit blocks whose targets are not the lowest physical qubits are first
    gathered there (one relabelling pass) and then run on the tensor cores; mixed
    with 1-qubit gates and other blocks, against the oracle, in both modes."""
    rng = np.random.default_rng(n * 31 + len(blocks))
    Us = [haar(32, rng) for _ in blocks]
    psi = workloads.random_state(n, 700 + n)
    for mode in ("plain", "fused"):
        ctx = qk.Context("c64", mode)
        ctx.add_qubits(n)
        ctx.set_state(psi)
        ref = oracle.OracleState(n, psi=psi)
        for U, t in zip(Us, blocks):
            gid = ctx.define_gate_matrix(U)
            ctx.apply_gate(gid, list(t))
            ref.apply_matrix(U, list(t))
            ctx.apply_gate("u3", [t[0]], params=[0.4, 1.1, 2.3])
            ref.apply_matrix(oracle.u3(0.4, 1.1, 2.3), [t[0]])
            ctx.apply_gate("z", [t[1]], controls=[(t[1] + 1) % n if (t[1] + 1) % n not in t else (t[1] + 2) % n])
            c = (t[1] + 1) % n if (t[1] + 1) % n not in t else (t[1] + 2) % n
            ref.apply_matrix(oracle.GATES_1Q["z"], [t[1]], [c])
        got = ctx.get_state().astype(np.complex128)
        err = float(np.max(np.abs(got - ref.psi)))
        assert err <= 1e-5, (mode, err)
        ctx.close()


@pytest.mark.parametrize("targets", [(4, 3, 2, 1, 0), (21, 6, 13, 2, 17)])
def test_block_tc_many_tiles_per_cta_matches_oracle(qk, targets):
    """24 qubits: 2^19 group rows, 4096 tiles of 128 rows, about 27 per persistent
    CTA, so every stage of the tile ring and both accumulators are reused many
    times; two blocks in a row against the oracle."""
    n = 24
    rng = np.random.default_rng(2400 + targets[0])
    U = haar(32, rng)
    psi = workloads.random_state(n, 2401)
    ctx = qk.Context("c64", "plain")
    ctx.add_qubits(n)
    ctx.set_state(psi)
    gid = ctx.define_gate_matrix(U)
    ctx.apply_gate(gid, list(targets))
    ctx.apply_gate(gid, list(targets))
    got = ctx.get_state().astype(np.complex128)
    ctx.close()
    ref = oracle.OracleState(n, psi=psi, openmp=True)
    ref.apply_matrix(U, list(targets))
    ref.apply_matrix(U, list(targets))
    err = float(np.max(np.abs(got - ref.psi)))
    assert err <= 1e-5, err


@pytest.mark.parametrize("n,targets", [(5, (2, 0, 4, 1)), (12, (4, 3, 2, 1)), (13, (9, 2, 11)), (17, (16, 3, 8, 12)),
                                       (20, (0, 1, 2))])
def test_three_and_four_qubit_blocks_on_tensor_cores(qk, n, targets):
    """3- and 4-qubit dense gates run as 5-qubit tensor-core blocks U (x) I (the
    spectator low qubits untouched), after a relabelling pass when their targets
    are not low; against the oracle and against the CUDA-core path."""
    k = len(targets)
    rng = np.random.default_rng(50 * n + k)
    U = haar(1 << k, rng)
    psi = workloads.random_state(n, 900 + n)
    got = {}
    for tc in (True, False):
        ctx = qk.Context("c64", "plain", tensor_cores=tc)
        ctx.add_qubits(n)
        ctx.set_state(psi)
        gid = ctx.define_gate_matrix(U)
        ctx.apply_gate(gid, list(targets))
        ctx.apply_gate("h", [targets[0]])
        ctx.apply_gate(gid, list(targets))
        got[tc] = ctx.get_state().astype(np.complex128)
        ctx.close()
    ref = oracle.OracleState(n, psi=psi)
    ref.apply_matrix(U, list(targets))
    ref.apply_matrix(oracle.GATES_1Q["h"], [targets[0]])
    ref.apply_matrix(U, list(targets))
    for tc in (True, False):
        err = float(np.max(np.abs(got[tc] - ref.psi)))
        assert err <= 1e-5, (tc, err)
