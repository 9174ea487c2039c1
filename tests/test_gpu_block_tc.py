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
