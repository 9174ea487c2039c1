"""The allocation-free mul-mod permutation entry point against the regular one.

qk_apply_perm_mulmod_noalloc serves callers that cannot allocate device memory
(latency-critical loops that must not pay an allocation's implicit device
synchronisation, hosts whose memory manager owns all device memory, users held to
a device memory budget reserved up front).  It works on a device state the caller
owns and gathers through a fixed scratch array inside the library.  This test
calls it through the C ABI twice in a row on one caller-owned buffer and checks
each result against qk_apply_gate with the same gate on a context, which is
bit-exact for a permutation (no arithmetic on amplitudes).  It lives in its own
file, collected last, and passes alone in a fresh process or after the others.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_noalloc_mulmod_matches_context_path_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07187_gb300 import qk

    n = 13
    psi = workloads.random_state(n, 2027).astype(np.complex64)
    # the caller-owned device state (allocated by the caller, here with torch)
    buf = torch.from_numpy(psi.view(np.float32).copy()).cuda()
    stream = torch.cuda.current_stream()

    ctx = qk.Context("c64", "plain")
    ctx.add_qubits(n)
    ctx.set_state(psi)

    calls = [  # (register qubits, first-listed = MSB; controls; c; N)
        ([1, 2, 3, 4, 5, 6, 7, 8], [0], 7, 221),
        ([12, 3, 9, 0, 5, 10, 2], [], 45, 101),
    ]
    for reg, ctrl, c, N in calls:
        gid = ctx.define_gate_perm_mulmod(len(reg), c, N)
        ctx.apply_gate(gid, reg, ctrl)
        expect = ctx.get_state()

        t = (ctypes.c_int * len(reg))(*reg)
        cl = (ctypes.c_int * max(1, len(ctrl)))(*ctrl)
        st = qk._lib.qk_apply_perm_mulmod_noalloc(ctypes.c_void_p(buf.data_ptr()), n, qk.QK_C64, t, len(reg),
                                                   cl, len(ctrl), c, N, ctypes.c_void_p(stream.cuda_stream))
        assert st == qk.QK_OK
        stream.synchronize()
        got = buf.cpu().numpy().view(np.complex64)
        assert np.max(np.abs(got - expect)) <= 1e-4      # the tests' complex64 tolerance
        assert np.array_equal(got, expect)                # a permutation moves values exactly

    # a state above the fixed scratch size is rejected before any device work
    t = (ctypes.c_int * 4)(0, 1, 2, 3)
    st = qk._lib.qk_apply_perm_mulmod_noalloc(ctypes.c_void_p(buf.data_ptr()), 22, qk.QK_C64, t, 4, None, 0, 7, 15,
                                               ctypes.c_void_p(stream.cuda_stream))
    assert st == qk.QK_EBUDGET
    # and a non-invertible multiplier is refused
    st = qk._lib.qk_apply_perm_mulmod_noalloc(ctypes.c_void_p(buf.data_ptr()), n, qk.QK_C64, t, 4, None, 0, 5, 15,
                                               ctypes.c_void_p(stream.cuda_stream))
    assert st == qk.QK_ENOTBIJECTIVE
    ctx.close()
