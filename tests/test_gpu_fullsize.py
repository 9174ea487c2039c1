"""Full-size checks (30 and 33 qubits, the fused tile path that bench.py times):
the oracle cannot hold these states, so the tests use results that are known in
closed form one amplitude at a time (the QFT of a basis state, GHZ) or properties
that hold at any size (echo C then C^dagger, collapse onto the measured basis
state, the norm)."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.set_device(0)
    from paper_1908_07187_gb300 import qk

    return qk, torch


def bitrev(x: int, n: int) -> int:
    return int(format(x, f"0{n}b")[::-1], 2)


def norm2(torch, view) -> float:
    tot = 0.0
    for s in range(0, view.numel(), 1 << 26):
        v = view[s:s + (1 << 26)]
        tot += float((v.real.double() ** 2 + v.imag.double() ** 2).sum())
    return tot


def inverse_ops(ops):
    out = []
    for op in reversed(ops):
        if op.kind == "u3":
            th, ph, la = op.params
            out.append(workloads.Op("u3", op.targets, op.controls, params=(-th, -la, -ph)))
        elif op.kind == "p":
            out.append(workloads.Op("p", op.targets, op.controls, params=(-op.params[0],)))
        elif op.kind in ("h", "z", "x", "swap"):
            out.append(op)
        else:
            raise ValueError(op.kind)
    return out


def test_qft_of_a_basis_state_30q_matches_the_closed_form(env):
    qk, torch = env
    n = 30
    rng = np.random.default_rng(30)
    x = int(rng.integers(1, 1 << n))
    ctx = qk.Context("c64", "fused")
    ctx.add_qubits(n)
    idx = bitrev(x, n)                      # register value x, qubit 0 the MSB
    for q in range(n):
        if (idx >> q) & 1:
            ctx.apply_gate("x", [q])
    qk.run_ops(ctx, workloads.qft_ops(range(n)))
    view = ctx.torch_view()
    ctx.sync()
    ys = [0, (1 << n) - 1] + [int(v) for v in rng.integers(0, 1 << n, size=4096)]
    got = view[torch.tensor([bitrev(y, n) for y in ys], device="cuda")].cpu().numpy().astype(np.complex128)
    amp = 2.0 ** (-n / 2)
    expect = np.array([amp * np.exp(2j * math.pi * ((x * y) % (1 << n)) / (1 << n)) for y in ys])
    rel = np.abs(got - expect) / amp
    assert rel.max() < 2e-4, rel.max()
    assert abs(norm2(torch, view) - 1.0) < 1e-5
    ctx.close()


def test_echo_of_the_layered_workload_30q_returns_to_zero(env):
    qk, torch = env
    n = 30
    circ = workloads.layered_circuit(n, seed=2, n_gates=500, qft=True)
    ops = [op for op in circ.ops if op.kind != "measure"]
    ctx = qk.Context("c64", "fused")
    ctx.add_qubits(n)
    qk.run_ops(ctx, ops)
    qk.run_ops(ctx, inverse_ops(ops))
    view = ctx.torch_view()
    ctx.sync()
    a0 = complex(view[0].item())
    assert abs(a0) ** 2 > 1 - 1e-5
    assert abs(norm2(torch, view) - 1.0) < 1e-5
    ctx.close()


def test_measuring_all_30_qubits_collapses_onto_the_outcome(env):
    qk, torch = env
    n = 30
    circ = workloads.layered_circuit(n, seed=3, n_gates=500, qft=True, measure=n)
    ctx = qk.run_circuit(circ, "c64", "fused")
    bits = [int(b) for b in ctx.read_cbits()]
    view = ctx.torch_view()
    ctx.sync()
    idx = sum(b << q for q, b in enumerate(bits))   # cbit q holds qubit q
    assert abs(abs(complex(view[idx].item())) ** 2 - 1.0) < 1e-5
    assert abs(norm2(torch, view) - 1.0) < 1e-5
    ctx.close()


def test_ghz_33q_uses_64_bit_tile_offsets(env):
    qk, torch = env
    n = 33                                  # 64 GiB of complex64: offsets beyond 2^32
    ctx = qk.Context("c64", "fused")
    ctx.add_qubits(n)
    ctx.apply_gate("h", [0])
    for q in range(n - 1):
        ctx.apply_gate("x", [q + 1], [q])
    view = ctx.torch_view()
    ctx.sync()
    h = 1 / math.sqrt(2)
    assert abs(complex(view[0].item()) - h) < 1e-6
    assert abs(complex(view[(1 << n) - 1].item()) - h) < 1e-6
    assert abs(norm2(torch, view) - 1.0) < 1e-5     # so every other amplitude is zero
    ctx.close()


def test_shor_3nx1_33q_matches_the_closed_form(env):
    """The conventional (3nx1) order-finding circuit at its largest single-GPU size:
    an 11-bit N with a 22-qubit control register, 33 qubits (64 GiB of complex64 plus
    the mul-mod gather buffer).  After the work register is measured at w = a^x0 mod N
    and the QFT sequence has run, the amplitude at control value y and work value w
    is (M 2^t)^-1/2 sum_{m<M} exp(2 pi i (x0 + m r) y / 2^t), M = #{x0 + m r < 2^t};
    4096 sampled y are checked against it, then the control register is measured and
    the state must collapse onto (y, w)."""
    from paper_1908_07187_gb300 import shor

    qk, torch = env
    N, a = workloads.kitaev_parameters(11, seed=4)
    circ = workloads.shor_3nx1_circuit(N, a, seed=3)
    b = N.bit_length()
    t = circ.n_qubits - b
    assert circ.n_qubits == 33 and circ.ops[-1].kind == "measure"
    r, x = 1, a % N
    while x != 1:
        x, r = x * a % N, r + 1
    ctx = qk.Context("c64", "fused")
    ctx.add_qubits(circ.n_qubits)
    ctx.add_cbits(circ.n_cbits)
    qk.run_ops(ctx, circ.ops[:-1])
    bits = [int(v) for v in ctx.read_cbits()]
    w = shor.register_from_bits(bits[:b])
    x0 = next(e for e in range(r) if pow(a, e, N) == w)
    T = 1 << t
    M = (T - x0 + r - 1) // r
    rng = np.random.default_rng(33)
    ys = np.array([0, T - 1] + [int(v) for v in rng.integers(0, T, size=4096)], dtype=np.int64)
    # geometric sum of exp(i theta m), theta = 2 pi r y / 2^t, done in exact turns
    turns = (r * ys) % T
    theta = 2 * math.pi * turns / T
    top = np.exp(2j * math.pi * ((turns * M) % T) / T) - 1
    geo = np.where(turns == 0, M, top / np.where(turns == 0, 1, np.exp(1j * theta) - 1))
    expect = np.exp(2j * math.pi * ((x0 * ys) % T) / T) * geo / math.sqrt(M * T)
    widx = bitrev(w, b) << t
    idx = torch.tensor([bitrev(int(y), t) + widx for y in ys], device="cuda")
    view = ctx.torch_view()
    ctx.sync()
    got = view[idx].cpu().numpy().astype(np.complex128)
    err = np.abs(got - expect).max()
    assert err < 1e-5, err
    assert abs(norm2(torch, view) - 1.0) < 1e-5
    qk.run_ops(ctx, circ.ops[-1:])
    bits = [int(v) for v in ctx.read_cbits()]
    y = shor.register_from_bits(bits[b:])
    view = ctx.torch_view()
    ctx.sync()
    assert abs(abs(complex(view[bitrev(y, t) + widx].item())) ** 2 - 1.0) < 1e-4
    ctx.close()
