"""Edge cases of the engine on the GPU: the smallest states, empty gate lists,
the fused planner's boundary at the tile width, degenerate measurements, and
argument errors that must leave the state unchanged."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qk():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.set_device(0)
    from paper_1908_07187_gb300 import qk as mod

    return mod


@pytest.mark.parametrize("mode", ["plain", "fused"])
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_one_qubit_state(qk, mode, prec):
    ctx = qk.Context(prec, mode)
    ctx.add_qubits(1)
    got0 = ctx.get_state()
    assert np.array_equal(got0, np.array([1, 0], dtype=got0.dtype))
    ctx.apply_gate("h", [0])
    ctx.apply_gate("t", [0])
    ref = oracle.OracleState(1)
    ref.apply_matrix(oracle.GATES_1Q["h"], [0])
    ref.apply_matrix(oracle.GATES_1Q["t"], [0])
    np.testing.assert_allclose(ctx.get_state(), ref.psi, atol=1e-6 if prec == "c64" else 1e-13)
    ctx.close()


def test_empty_gate_list_and_flush(qk):
    ctx = qk.Context("c64", "fused")
    ctx.add_qubits(14)
    qk.run_ops(ctx, [])
    ctx.flush()
    st = ctx.get_state()
    assert st[0] == 1 and np.count_nonzero(st) == 1
    ctx.close()


@pytest.mark.parametrize("n", [12, 13, 14])
def test_fused_planner_at_the_tile_width(qk, n):
    # below 13 qubits the fused mode runs gate by gate; at 13 one tile is the state
    circ = workloads.layered_circuit(n, seed=8, n_gates=120)
    ref = oracle.run_circuit(circ)
    ctx = qk.run_circuit(circ, "c64", "fused")
    np.testing.assert_allclose(ctx.get_state(), ref.psi, atol=1e-4)
    ctx.close()


def test_measuring_a_basis_state_is_certain(qk):
    # P0 is exactly 0 or 1: the outcome does not depend on the uniform
    for u in (0.0, 0.5, 0.999999):
        ctx = qk.Context("c64", "fused")
        ctx.add_qubits(15)
        ctx.add_cbits(2)
        ctx.apply_gate("x", [3])
        ctx.measure([3, 4], [u, u], [0, 1], wait=True)
        assert list(ctx.read_cbits()) == [1, 0]
        st = ctx.get_state()
        assert abs(st[1 << 3]) == pytest.approx(1.0)
        ctx.close()


def test_rejected_gate_leaves_the_state_unchanged(qk):
    psi = workloads.random_state(6, 3)
    ctx = qk.Context("c128", "plain")
    ctx.add_qubits(6)
    ctx.set_state(psi)
    for bad in (lambda: ctx.apply_gate("h", [6]),                 # qubit out of range
                lambda: ctx.apply_gate("x", [2], [2]),            # control equals target
                lambda: ctx.apply_gate("u3", [1], params=[0.1]),  # missing parameters
                lambda: ctx.measure([0], [1.5])):                 # uniform outside [0, 1)
        with pytest.raises(qk.QKError) as e:
            bad()
        assert e.value.status == qk.QK_EINVAL
    np.testing.assert_array_equal(ctx.get_state(), psi)
    ctx.close()


def test_bounded_wait_timeout_is_reported_and_context_stays_usable(qk):
    """The bounded device-side wait gives up (the self-test waits on a barrier
    nothing arrives at), qk_sync reports QK_ETIMEOUT once, and the context keeps
    working: the state is untouched and later gates are correct."""
    import oracle

    n = 6
    psi = workloads.random_state(n, 71)
    ctx = qk.Context("c64", "fused")
    ctx.add_qubits(n)
    ctx.set_state(psi)
    ctx.selftest_timeout()
    with pytest.raises(qk.QKError) as e:
        ctx.sync()
    assert e.value.status == qk.QK_ETIMEOUT
    ctx.sync()                                   # the condition was cleared
    ctx.apply_gate("h", [2])
    ref = oracle.OracleState(n, psi=psi)
    ref.apply_matrix(oracle.GATES_1Q["h"], [2])
    np.testing.assert_allclose(ctx.get_state(), ref.psi, atol=1e-5)
    ctx.close()


def test_freed_state_memory_is_reused(qk):
    """The library keeps freed device memory in its own pool for reuse (and trims
    it when its last context or batch goes): creating and destroying a 2 GiB state
    three times holds at most one such block, never three."""
    import torch

    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        ctx = qk.Context("c64", "fused")
        ctx.add_qubits(28)
        ctx.apply_gate("h", [27])
        ctx.sync()
        ctx.close()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < int(2.5 * 2**30), (free0, free1)
