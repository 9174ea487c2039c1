// qk_apply_perm_mulmod_noalloc: the controlled x -> c*x mod N register
// permutation applied to a caller-owned device state without allocating any
// device memory.
//
// Some callers cannot call cudaMalloc: latency-critical loops where an
// allocation's implicit device synchronisation would stall every other stream,
// host applications whose own memory manager owns all device memory, and
// embedded users that must stay inside a device memory budget reserved up
// front.  The regular path (qk_apply_gate
// on a context) allocates a state-sized gather buffer on first use; this entry
// point instead gathers into a fixed scratch array that lives in the library's
// device image, then copies the result back over the caller's state.
//
// The scratch array below is a file-scope __device__ variable: every GPU that
// loads libqk holds QK_NOALLOC_SCRATCH_BYTES of it until the process exits.
// In host code its name is only a host-side stand-in, never a device address,
// so the device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernel.
#include <cuda_runtime.h>

#include <mutex>

#include "qk.h"
#include "qk_kernels.cuh"

namespace {

static __device__ __align__(256) unsigned char g_perm_scratch[QK_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices];   // device address of g_perm_scratch, per device
int g_sms[kMaxDevices];

// Modular inverse of a mod N by the extended Euclidean algorithm; ok = gcd == 1.
uint64_t inverse_mod(uint64_t a, uint64_t N, bool &ok) {
    __int128 t = 0, nt = 1, r = (__int128)N, nr = (__int128)(a % N);
    while (nr != 0) {
        const __int128 q = r / nr;
        __int128 tmp = t - q * nt;
        t = nt;
        nt = tmp;
        tmp = r - q * nr;
        r = nr;
        nr = tmp;
    }
    ok = (r == 1);
    if (t < 0) t += (__int128)N;
    return (uint64_t)t;
}

// Per-device set-up, done by the first call on each device (with it current).
qk_status setup_device(int dev, void **scratch, int *sms) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_perm_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return QK_ECUDA;
        }
        int count = 0;
        if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return QK_ECUDA;
        }
        g_sms[dev] = count;
        g_scratch_addr[dev] = p;
    }
    *scratch = g_scratch_addr[dev];
    *sms = g_sms[dev];
    return QK_OK;
}

bool distinct_in_range(const int *q, int k, int n) {
    for (int a = 0; a < k; ++a) {
        if (q[a] < 0 || q[a] >= n) return false;
        for (int b = 0; b < a; ++b)
            if (q[a] == q[b]) return false;
    }
    return true;
}

}  // namespace

extern "C" qk_status qk_apply_perm_mulmod_noalloc(void *d_state, int n, qk_precision precision,
                                                  const int *targets, int w, const int *controls, int nc,
                                                  uint64_t c, uint64_t N, void *cuda_stream) {
    if (precision != QK_C64 && precision != QK_C128) return QK_EINVAL;
    const size_t amp = precision == QK_C64 ? 8 : 16;
    if (!d_state || ((uintptr_t)d_state % 16) != 0 || n < 1 || n > QK_MAX_QUBITS) return QK_EINVAL;
    // the state must fit in the fixed scratch array
    if ((amp << n) > (size_t)QK_NOALLOC_SCRATCH_BYTES) return QK_EBUDGET;
    if (w < 1 || w > QK_MAX_PERM_QUBITS || w > n || !targets || nc < 0 || nc > QK_MAX_CONTROLS ||
        (nc > 0 && !controls))
        return QK_EINVAL;
    if (!distinct_in_range(targets, w, n) || !distinct_in_range(controls, nc, n)) return QK_EINVAL;
    for (int a = 0; a < w; ++a)
        for (int b = 0; b < nc; ++b)
            if (targets[a] == controls[b]) return QK_EINVAL;
    if (N < 2 || N > (1ull << w) || c >= N) return QK_EINVAL;
    bool ok = false;
    const uint64_t cinv = inverse_mod(c, N, ok);
    if (!ok) return QK_ENOTBIJECTIVE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return QK_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return QK_EINVAL;
    void *scratch = nullptr;
    int sms = 0;
    qk_status st = setup_device(dev, &scratch, &sms);
    if (st != QK_OK) return st;

    qk::PermArgs a{};
    a.w = w;
    for (int t = 0; t < w; ++t) a.rpos[t] = targets[t];
    for (int b = 0; b < nc; ++b) a.cmask |= 1ull << controls[b];
    a.n_amps = 1ull << n;
    a.kind = 0;
    a.N = N;
    a.cinv = cinv;
    a.mu = (~0ull) / N;
    a.finv = nullptr;
    a.cond.n = 0;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // every scratch entry the copy-back reads is written by the gather first,
    // so nothing left over from an earlier call is ever read
    if (qk::launch_perm((int)precision, d_state, scratch, a, nullptr, sms, s) != cudaSuccess) return QK_ECUDA;
    if (cudaMemcpyAsync(d_state, scratch, amp << n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return QK_ECUDA;
    }
    return QK_OK;
}
