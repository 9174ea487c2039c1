// K8: many small circuits in one launch.
//
// A circuit of n <= 13 qubits fits in shared memory (2^13 complex64 = 64 KiB),
// so one CTA can run the whole circuit -- 2x2 gates with quantum controls,
// diagonal gates, the controlled mul-mod oracle, mid-circuit measurements and
// classically conditioned gates -- without touching HBM between gates.  A batch
// launch gives every circuit its own CTA; the circuits are independent and may
// differ in size and gate list.  This is the shared launch that serving uses for
// small requests (one launch per batch instead of one launch per gate).
//
// Semantics match the per-gate engine op for op: measurement is one qubit at a
// time in list order, P0 summed in FP64 over the (renormalised) state, outcome
// 1 iff u >= P0, collapse and renormalise; cbits start at 0.
//
// Circuits of 14..24 qubits (unitary gates with at most one control) keep their
// states in HBM: each is planned into fused tile passes on the host (in
// parallel over the host's cores), and pass k of every such circuit runs in one
// batched tile launch (k_tile_batch), so a batch of thousands of circuits costs
// one launch per pass index rather than one per circuit pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "qk.h"
#include "qk_host.h"
#include "qk_kernels.cuh"
#include "qk_plan.h"

namespace qk {
namespace {

constexpr int kBThreads = 256;
constexpr int kBMaxQubits = 13;
constexpr int kBMaxCbits = 64;
constexpr int kBMaxLargeQubits = 24;
constexpr int kOpChunk = kBThreads * 16 / 64;   // ops staged per chunk: one 16-byte word per thread

// B_RAW never reaches the device: a 1-target built-in gate that is never diagonal,
// kept as its id and angles until qk_batch_run forms its matrix (as B_U2).
enum BOpKind : uint8_t { B_U2 = 0, B_PHASE = 1, B_MULMOD = 2, B_MEASURE = 3, B_RAW = 0x40 };

// One op of a small-circuit program (64 bytes).
struct BOp {
    uint8_t kind, q, ncond, w;
    uint8_t cond[4];
    uint32_t cmask, val;       // controls (U2, MULMOD) / phase mask and value
    union {
        float m[8];            // U2: m00, m01, m10, m11 (re, im)
        struct {
            float re, im;      // PHASE factor
        } ph;
        struct {
            uint32_t N, cinv;  // MULMOD: y -> cinv*y mod N gives the source register value
            uint8_t rpos[16];  // register qubits, rpos[0] = MSB
        } mm;
        struct {
            double u;          // MEASURE uniform
            int32_t dest;      // destination cbit (-1: none)
        } ms;
        struct {
            double p[3];       // RAW: the built-in's parameters
            int32_t id, np;    // its gate id and parameter count
        } raw;
    };
    uint8_t pad[16];
};
static_assert(sizeof(BOp) == 64, "BOp layout");

struct BCirc {
    uint32_t op_begin, op_end;
    uint32_t n, ncb;
    uint32_t cb_off;
    uint32_t flags;            // bit 0: holds a mul-mod (needs the second state buffer)
    uint64_t state_off;        // in amplitudes
};

__device__ __forceinline__ uint32_t ins0(uint32_t j, int pos) {
    const uint32_t lo = j & ((1u << pos) - 1);
    return ((j - lo) << 1) | lo;
}

// K consecutive uncontrolled 2x2 gates on distinct qubits qs[0..K-1] (in program
// order, matrices in gops[0..K-1]): each thread takes groups of 2^K amplitudes that
// differ in those qubits, applies the K gates in registers and writes the group
// back once, so the state crosses shared memory once per K gates instead of once
// per gate.
template <int K>
__device__ __forceinline__ void u2_group(float2 *A, uint32_t dim, const BOp *gops, const int *qs) {
    int qsort[K];
#pragma unroll
    for (int j = 0; j < K; ++j) qsort[j] = qs[j];
#pragma unroll
    for (int a = 1; a < K; ++a)
#pragma unroll
        for (int b = a; b > 0; --b)
            if (qsort[b] < qsort[b - 1]) {
                const int t = qsort[b];
                qsort[b] = qsort[b - 1];
                qsort[b - 1] = t;
            }
    uint32_t off[1 << K];
    off[0] = 0;
#pragma unroll
    for (int r = 1; r < (1 << K); ++r) off[r] = off[r & (r - 1)] + (1u << qs[__ffs(r) - 1]);
    for (uint32_t g = threadIdx.x; g < (dim >> K); g += kBThreads) {
        uint32_t base = g;
#pragma unroll
        for (int j = 0; j < K; ++j) base = ins0(base, qsort[j]);
        float2 x[1 << K];
#pragma unroll
        for (int r = 0; r < (1 << K); ++r) x[r] = A[base + off[r]];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const float *m = gops[j].m;
            const float2 m00 = make_float2(m[0], m[1]), m01 = make_float2(m[2], m[3]);
            const float2 m10 = make_float2(m[4], m[5]), m11 = make_float2(m[6], m[7]);
#pragma unroll
            for (int r = 0; r < (1 << K); ++r) {
                if (r & (1 << j)) continue;
                const float2 a = x[r], b = x[r | (1 << j)];
                x[r] = make_float2(m00.x * a.x - m00.y * a.y + m01.x * b.x - m01.y * b.y,
                                   m00.x * a.y + m00.y * a.x + m01.x * b.y + m01.y * b.x);
                x[r | (1 << j)] = make_float2(m10.x * a.x - m10.y * a.y + m11.x * b.x - m11.y * b.y,
                                              m10.x * a.y + m10.y * a.x + m11.x * b.y + m11.y * b.x);
            }
        }
#pragma unroll
        for (int r = 0; r < (1 << K); ++r) A[base + off[r]] = x[r];
    }
}

__global__ void __launch_bounds__(kBThreads) k_batch(const BCirc *__restrict__ circs, const BOp *__restrict__ ops,
                                                     float2 *__restrict__ states, uint8_t *__restrict__ cbits_out,
                                                     int store_state) {
    extern __shared__ __align__(16) unsigned char sm[];
    const BCirc c = circs[blockIdx.x];
    const int n = (int)c.n;
    const uint32_t dim = 1u << n;
    __shared__ double red[2][kBThreads / 32];
    __shared__ uint8_t cb[kBMaxCbits];
    __shared__ int s_m;
    __shared__ float s_scale;
    __shared__ __align__(16) BOp s_ops[2][kOpChunk];
    float2 *A = reinterpret_cast<float2 *>(sm);
    float2 *B = A + dim;
    const int tid = threadIdx.x;
    for (uint32_t i = tid; i < dim; i += kBThreads) A[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
    for (int k = tid; k < kBMaxCbits; k += kBThreads) cb[k] = 0;
    __syncthreads();

    // the program streams through shared memory in chunks of kOpChunk ops (one
    // 16-byte load per thread per chunk); the next chunk's load is issued before
    // the current chunk runs, so its latency hides behind the gates
    const uint32_t nops = c.op_end - c.op_begin;
    const uint4 *gops = reinterpret_cast<const uint4 *>(ops + c.op_begin);
    const uint32_t nwords = nops * (uint32_t)(sizeof(BOp) / 16);
    if ((uint32_t)tid < nwords) reinterpret_cast<uint4 *>(s_ops[0])[tid] = gops[tid];
    __syncthreads();
    for (uint32_t chunk = 0; chunk * kOpChunk < nops; ++chunk) {
        const int buf = (int)(chunk & 1);
        const uint32_t nw = (chunk + 1) * kOpChunk * (uint32_t)(sizeof(BOp) / 16) + (uint32_t)tid;
        uint4 next = make_uint4(0, 0, 0, 0);
        if (nw < nwords) next = gops[nw];
        const uint32_t cnt = min((uint32_t)kOpChunk, nops - chunk * kOpChunk);
        for (uint32_t oi = 0; oi < cnt; ++oi) {
            const BOp &op = s_ops[buf][oi];
            bool act = true;
            for (int k = 0; k < op.ncond; ++k) act = act && cb[op.cond[k]] != 0;
            if (op.kind == B_U2 && op.ncond == 0 && op.cmask == 0) {
                // two consecutive uncontrolled, unconditioned 2x2 gates on distinct
                // qubits within this chunk are applied as one register group (groups
                // of 3 and 4 measured slower: their registers cut the CTAs per SM)
                int qs[2] = {op.q, 0};
                int k = 1;
                while (k < 2 && oi + k < cnt) {
                    const BOp &nx = s_ops[buf][oi + k];
                    bool ok = nx.kind == B_U2 && nx.ncond == 0 && nx.cmask == 0;
                    for (int j = 0; j < k && ok; ++j) ok = qs[j] != nx.q;
                    if (!ok) break;
                    qs[k++] = nx.q;
                }
                if (k == 2) u2_group<2>(A, dim, &op, qs);
                else u2_group<1>(A, dim, &op, qs);
                oi += (uint32_t)(k - 1);
            } else if (op.kind == B_U2) {
                if (act) {
                    const float2 m00 = make_float2(op.m[0], op.m[1]), m01 = make_float2(op.m[2], op.m[3]);
                    const float2 m10 = make_float2(op.m[4], op.m[5]), m11 = make_float2(op.m[6], op.m[7]);
                    for (uint32_t p = tid; p < (dim >> 1); p += kBThreads) {
                        const uint32_t i0 = ins0(p, op.q), i1 = i0 | (1u << op.q);
                        if ((i0 & op.cmask) != op.cmask) continue;
                        const float2 a = A[i0], b = A[i1];
                        A[i0] = make_float2(m00.x * a.x - m00.y * a.y + m01.x * b.x - m01.y * b.y,
                                            m00.x * a.y + m00.y * a.x + m01.x * b.y + m01.y * b.x);
                        A[i1] = make_float2(m10.x * a.x - m10.y * a.y + m11.x * b.x - m11.y * b.y,
                                            m10.x * a.y + m10.y * a.x + m11.x * b.y + m11.y * b.x);
                    }
                }
            } else if (op.kind == B_PHASE) {
                if (act) {
                    // only the matching amplitudes: u enumerates the bits outside the
                    // mask, a zero goes in at each mask bit, then the required values
                    const float fr = op.ph.re, fi = op.ph.im;
                    const uint32_t cnt = dim >> __popc(op.cmask);
                    for (uint32_t u = tid; u < cnt; u += kBThreads) {
                        uint32_t i = u;
                        for (uint32_t m = op.cmask; m; m &= m - 1) i = ins0(i, __ffs(m) - 1);
                        i |= op.val;
                        const float2 a = A[i];
                        A[i] = make_float2(a.x * fr - a.y * fi, a.x * fi + a.y * fr);
                    }
                }
            } else if (op.kind == B_MULMOD) {
                for (uint32_t i = tid; i < dim; i += kBThreads) {
                    uint32_t src = i;
                    if (act && (i & op.cmask) == op.cmask) {
                        uint32_t y = 0;
                        for (int b = 0; b < op.w; ++b) y = (y << 1) | ((i >> op.mm.rpos[b]) & 1u);
                        if (y < op.mm.N) {
                            const uint32_t x = (uint32_t)(((uint64_t)op.mm.cinv * y) % op.mm.N);
                            for (int b = 0; b < op.w; ++b) {
                                const uint32_t bit = (x >> (op.w - 1 - b)) & 1u;
                                src = (src & ~(1u << op.mm.rpos[b])) | (bit << op.mm.rpos[b]);
                            }
                        }
                    }
                    B[i] = A[src];
                }
                __syncthreads();
                float2 *t = A;
                A = B;
                B = t;
            } else {  // B_MEASURE on qubit q
                // |a|^2 in FP32 into compensated float pairs (GB300 has 2 FP64 lanes per
                // SM per clock), FP64 from the per-thread sums on
                FSum g0, g1;
                for (uint32_t i = tid; i < dim; i += kBThreads) {
                    const float2 a = A[i];
                    const float pa = a.x * a.x + a.y * a.y;
                    if ((i >> op.q) & 1u) g1.add(pa); else g0.add(pa);
                }
                double d0 = g0.value(), d1 = g1.value();
                for (int o = 16; o > 0; o >>= 1) {
                    d0 += __shfl_xor_sync(0xffffffffu, d0, o);
                    d1 += __shfl_xor_sync(0xffffffffu, d1, o);
                }
                if ((tid & 31) == 0) {
                    red[0][tid >> 5] = d0;
                    red[1][tid >> 5] = d1;
                }
                __syncthreads();
                if (tid == 0) {
                    double s0 = 0.0, s1 = 0.0;
                    for (int w = 0; w < kBThreads / 32; ++w) {
                        s0 += red[0][w];
                        s1 += red[1][w];
                    }
                    const double tot = s0 + s1;
                    const double p0 = tot > 0.0 ? s0 / tot : 1.0;
                    const int m = (op.ms.u >= p0) ? 1 : 0;
                    const double pm = m ? s1 : s0;
                    s_m = m;
                    s_scale = (float)(pm > 0.0 ? 1.0 / sqrt(pm) : 0.0);
                    if (op.ms.dest >= 0) cb[op.ms.dest] = (uint8_t)m;
                }
                __syncthreads();
                const int m = s_m;
                const float sc = s_scale;
                for (uint32_t i = tid; i < dim; i += kBThreads) {
                    const float k = ((int)((i >> op.q) & 1u) == m) ? sc : 0.f;
                    const float2 a = A[i];
                    A[i] = make_float2(a.x * k, a.y * k);
                }
            }
            __syncthreads();
        }
        if (nw < nwords) reinterpret_cast<uint4 *>(s_ops[buf ^ 1])[tid] = next;
        __syncthreads();
    }
    for (uint32_t k = tid; k < c.ncb; k += kBThreads) cbits_out[c.cb_off + k] = cb[k];
    if (store_state)
        for (uint32_t i = tid; i < dim; i += kBThreads) states[c.state_off + i] = A[i];
}

// |0...0> for each listed state of the large-circuit pool (the pool is zeroed first)
__global__ void k_set_basis0(float2 *pool, const uint64_t *offs, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) pool[offs[i]] = make_float2(1.f, 0.f);
}

}  // namespace
}  // namespace qk

// ===========================================================================
// host side
// ===========================================================================
struct qk_batch {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    bool pool_held = false;   // holds the library's memory pool of its device
    int sms = 148;
    std::vector<qk::BOp> ops;
    std::vector<qk::BCirc> circs;
    uint64_t total_amps = 0;
    uint32_t total_cb = 0;
    int max_n = 0;
    // device buffers (grown as needed)
    qk::BOp *d_ops = nullptr;
    size_t cap_ops = 0;
    qk::BCirc *d_circs = nullptr;
    size_t cap_circs = 0;
    float2 *d_states = nullptr;
    size_t cap_states = 0;
    uint8_t *d_cbits = nullptr;
    size_t cap_cbits = 0;
    // pinned staging for the uploads (valid until the next run)
    void *h_stage = nullptr;
    size_t cap_stage = 0;
    cudaEvent_t done = nullptr;
    cudaEvent_t start = nullptr;       // recorded once the host work of a run is done
    bool start_recorded = false;
    bool store_state = true;
    std::string err;
    // circuits of 14..24 qubits: gate lists for the tile planner, states in HBM
    struct Large {
        int circ;                      // index in circs
        int n;
        // its gates as validated list entries (physical qubit = qubit, no
        // relabelling); the planning threads turn them into planner ops
        std::vector<qk_gate_op> gates;
        uint64_t state_off = 0;        // in the large-state pool, amplitudes
        int npasses = 0;
    };
    std::vector<Large> large;
    std::vector<int> large_of;         // circuit index -> index in large (-1: small)
    uint64_t large_amps = 0;
    float2 *d_lstates = nullptr;
    size_t cap_lstates = 0;
    qk::TileProg *d_lprogs = nullptr;
    size_t cap_lprogs = 0;
    uint32_t *d_lfirst = nullptr;
    size_t cap_lfirst = 0;
    uint64_t *d_loffs = nullptr;
    size_t cap_loffs = 0;
    qk::TileOp *d_lops = nullptr;
    size_t cap_lops = 0;
    qk::LayerGate *d_llg = nullptr;
    size_t cap_llg = 0;
    qk::LinTerm *d_llin = nullptr;
    size_t cap_llin = 0;
    double plan_ms = 0.0;              // host planning time of the last run
    int large_launches = 0;            // batched tile launches of the last run
};

namespace {

qk_status bfail(qk_batch *b, qk_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    return s;
}

bool cur_circuit(qk_batch *b, qk::BCirc **c) {
    if (b->circs.empty()) return false;
    *c = &b->circs.back();
    return true;
}

// Device buffers are stream-ordered on the batch's stream (the library's pool):
// growing one does not synchronise the device while other streams run.
template <typename T>
qk_status grow(qk_batch *b, T **p, size_t *cap, size_t need) {
    if (need <= *cap) return QK_OK;
    size_t nc = std::max(need, *cap * 2);
    if (*p) cudaFreeAsync(*p, b->stream);
    *p = nullptr;
    *cap = 0;
    if (qk::pool_malloc((void **)p, sizeof(T) * nc, b->device, b->stream) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, QK_ENOMEM, "batch: cannot allocate %zu bytes", sizeof(T) * nc);
    }
    *cap = nc;
    return QK_OK;
}

bool fill_cond(qk::BOp &op, const qk::BCirc &c, const int *cond, int ncc) {
    if (ncc < 0 || ncc > 4 || (ncc > 0 && !cond)) return false;
    op.ncond = (uint8_t)ncc;
    for (int k = 0; k < ncc; ++k) {
        if (cond[k] < 0 || cond[k] >= (int)c.ncb) return false;
        op.cond[k] = (uint8_t)cond[k];
    }
    return true;
}

bool distinct(const int *q, int k, int n) {
    for (int a = 0; a < k; ++a) {
        if (q[a] < 0 || q[a] >= n) return false;
        for (int b2 = 0; b2 < a; ++b2)
            if (q[a] == q[b2]) return false;
    }
    return true;
}

// The B_RAW ops of the small circuits as B_U2 (their matrices in FP64, stored as
// FP32), split over the host's cores for long lists.
void form_raw_ops(std::vector<qk::BOp> &ops) {
    const size_t n = ops.size();
    auto work = [&ops](size_t lo, size_t hi) {
        for (size_t i = lo; i < hi; ++i) {
            qk::BOp &op = ops[i];
            if (op.kind != qk::B_RAW) continue;
            const double p[3] = {op.raw.p[0], op.raw.p[1], op.raw.p[2]};
            const int id = op.raw.id, np = op.raw.np;
            qk::cd m[4];
            int ntg = 0;
            qk::builtin_matrix(id, p, np, m, ntg);
            op.kind = qk::B_U2;
            for (int e = 0; e < 4; ++e) {
                op.m[2 * e] = (float)m[e].real();
                op.m[2 * e + 1] = (float)m[e].imag();
            }
        }
    };
    const size_t nth = n < (1u << 16) ? 1 : std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (nth == 1) {
        work(0, n);
        return;
    }
    std::vector<std::thread> th;
    for (size_t t = 0; t < nth; ++t) th.emplace_back(work, n * t / nth, n * (t + 1) / nth);
    for (auto &t : th) t.join();
}

// A validated gate of a circuit above 13 qubits (one target, at most one control,
// no classical condition) as planner ops: a 2x2 op, or one phase op per diagonal
// entry that is not 1.
void append_fused(std::vector<qk::FusedOp> &out, const qk_gate_op &g) {
    qk::cd m[4];
    int ntg = 0;
    qk::builtin_matrix(g.gate_id, g.params, g.np, m, ntg);
    const uint64_t cmask = g.nc ? 1ull << g.controls[0] : 0ull;
    const int q = g.target;
    if (m[1] == 0.0 && m[2] == 0.0) {
        for (int e = 0; e < 2; ++e) {
            const qk::cd f = e ? m[3] : m[0];
            if (f == 1.0) continue;
            qk::FusedOp o;
            o.kind = qk::FusedOp::PHASE;
            o.mask = cmask | (1ull << q);
            o.val = cmask | (e ? (1ull << q) : 0ull);
            o.f = f;
            out.push_back(o);
        }
    } else {
        qk::FusedOp o;
        o.kind = qk::FusedOp::U2;
        o.q = q;
        o.cmask = cmask;
        for (int e = 0; e < 4; ++e) o.m[e] = m[e];
        out.push_back(o);
    }
}

// The circuits above 13 qubits: plan each into tile passes (host threads), pack
// the pass programs into device pools ordered by pass index, set the states to
// |0...0> and launch pass k of every circuit that has one in one batched launch.
qk_status run_large(qk_batch *b) {
    const auto t0 = std::chrono::steady_clock::now();
    struct Plan {
        std::vector<qk::TileProg> progs;
        std::vector<qk::TileOp> ops;
        std::vector<qk::LayerGate> lg;
        std::vector<qk::LinTerm> lin;
        qk_status st = QK_OK;
        std::string err;
    };
    const int nl = (int)b->large.size();
    std::vector<Plan> plans(nl);
    const int nth = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::atomic<int> next(0);
    auto worker = [&]() {
        qk::TilePlanner *pl = qk::make_planner();
        std::vector<qk::FusedOp> fops;
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= nl) break;
            const auto &L = b->large[i];
            Plan &out = plans[i];
            fops.clear();
            fops.reserve(L.gates.size());
            for (const qk_gate_op &g : L.gates) append_fused(fops, g);
            const qk::PassSink sink = [&](qk::TileParams &P) -> qk_status {
                if (P.n_conds > 0) {   // unreachable: large circuits take no classical conditions
                    out.err = "batch: classical conditions are not batched above 13 qubits";
                    return QK_EINVAL;
                }
                qk::TileProg h{};
                static_cast<qk::TileHead &>(h) = P;
                h.op0 = (uint32_t)out.ops.size();
                h.lg0 = (uint32_t)out.lg.size();
                h.lin0 = (uint32_t)out.lin.size();
                out.ops.insert(out.ops.end(), P.ops, P.ops + P.nops);
                out.lg.insert(out.lg.end(), P.lg, P.lg + P.nlg);
                out.lin.insert(out.lin.end(), P.lin, P.lin + P.nlin);
                out.progs.push_back(h);
                return QK_OK;
            };
            const char *err = "";
            out.st = qk::plan_passes(pl, L.n, fops, sink, &err);
            if (out.st != QK_OK && out.err.empty()) out.err = err;
        }
        qk::free_planner(pl);
    };
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t) th.emplace_back(worker);
    for (auto &t : th) t.join();
    size_t nops = 0, nlg = 0, nlin = 0, nprog = 0;
    int maxp = 0;
    std::vector<size_t> op_base(nl), lg_base(nl), lin_base(nl);
    for (int i = 0; i < nl; ++i) {
        if (plans[i].st != QK_OK) return bfail(b, plans[i].st, "batch: circuit %d: %s", b->large[i].circ, plans[i].err.c_str());
        op_base[i] = nops;
        lg_base[i] = nlg;
        lin_base[i] = nlin;
        nops += plans[i].ops.size();
        nlg += plans[i].lg.size();
        nlin += plans[i].lin.size();
        nprog += plans[i].progs.size();
        b->large[i].npasses = (int)plans[i].progs.size();
        maxp = std::max(maxp, b->large[i].npasses);
    }
    qk_status s;
    if ((s = grow(b, &b->d_lstates, &b->cap_lstates, std::max<uint64_t>(1, b->large_amps))) != QK_OK) return s;
    if ((s = grow(b, &b->d_lprogs, &b->cap_lprogs, std::max<size_t>(1, nprog))) != QK_OK) return s;
    if ((s = grow(b, &b->d_lfirst, &b->cap_lfirst, nprog + (size_t)maxp + 1)) != QK_OK) return s;
    if ((s = grow(b, &b->d_loffs, &b->cap_loffs, (size_t)nl)) != QK_OK) return s;
    if ((s = grow(b, &b->d_lops, &b->cap_lops, std::max<size_t>(1, nops))) != QK_OK) return s;
    if ((s = grow(b, &b->d_llg, &b->cap_llg, std::max<size_t>(1, nlg))) != QK_OK) return s;
    if ((s = grow(b, &b->d_llin, &b->cap_llin, std::max<size_t>(1, nlin))) != QK_OK) return s;
    // programs ordered by pass index; first[] splits each launch's grid
    std::vector<qk::TileProg> progs;
    progs.reserve(nprog);
    std::vector<uint32_t> first;
    std::vector<std::pair<size_t, size_t>> launch;   // (first program, first[] index)
    std::vector<uint32_t> ctas;
    for (int k = 0; k < maxp; ++k) {
        launch.push_back({progs.size(), first.size()});
        uint32_t acc = 0;
        for (int i = 0; i < nl; ++i) {
            if (k >= (int)plans[i].progs.size()) continue;
            qk::TileProg h = plans[i].progs[k];
            h.op0 += (uint32_t)op_base[i];
            h.lg0 += (uint32_t)lg_base[i];
            h.lin0 += (uint32_t)lin_base[i];
            h.psi = b->d_lstates + b->large[i].state_off;
            progs.push_back(h);
            first.push_back(acc);
            acc += (uint32_t)h.n_tiles;
        }
        first.push_back(acc);
        ctas.push_back(acc);
    }
    std::vector<qk::TileOp> ops;
    std::vector<qk::LayerGate> lg;
    std::vector<qk::LinTerm> lin;
    ops.reserve(nops);
    lg.reserve(nlg);
    lin.reserve(nlin);
    std::vector<uint64_t> offs(nl);
    for (int i = 0; i < nl; ++i) {
        ops.insert(ops.end(), plans[i].ops.begin(), plans[i].ops.end());
        lg.insert(lg.end(), plans[i].lg.begin(), plans[i].lg.end());
        lin.insert(lin.end(), plans[i].lin.begin(), plans[i].lin.end());
        offs[i] = b->large[i].state_off;
    }
    b->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (cudaEventRecord(b->start, b->stream) != cudaSuccess) return bfail(b, QK_ECUDA, "batch: event record failed");
    b->start_recorded = true;
    auto up = [&](void *dst, const void *src, size_t bytes) {
        return bytes == 0 || cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, b->stream) == cudaSuccess;
    };
    if (!up(b->d_lprogs, progs.data(), sizeof(qk::TileProg) * progs.size()) ||
        !up(b->d_lfirst, first.data(), sizeof(uint32_t) * first.size()) ||
        !up(b->d_loffs, offs.data(), sizeof(uint64_t) * offs.size()) ||
        !up(b->d_lops, ops.data(), sizeof(qk::TileOp) * ops.size()) ||
        !up(b->d_llg, lg.data(), sizeof(qk::LayerGate) * lg.size()) ||
        !up(b->d_llin, lin.data(), sizeof(qk::LinTerm) * lin.size()))
        return bfail(b, QK_ECUDA, "batch: program upload failed");
    if (cudaMemsetAsync(b->d_lstates, 0, sizeof(float2) * b->large_amps, b->stream) != cudaSuccess)
        return bfail(b, QK_ECUDA, "batch: state reset failed");
    qk::k_set_basis0<<<(nl + 255) / 256, 256, 0, b->stream>>>(b->d_lstates, b->d_loffs, nl);
    if (cudaGetLastError() != cudaSuccess) return bfail(b, QK_ECUDA, "batch: state reset failed");
    b->large_launches = 0;
    for (int k = 0; k < maxp; ++k) {
        const int np = (int)((k + 1 < maxp ? launch[k + 1].first : progs.size()) - launch[k].first);
        // the kernel instance without the general-op path when no program needs it
        bool general = false;
        for (int q = 0; q < np && !general; ++q) {
            const qk::TileProg &h = progs[launch[k].first + q];
            general = qk::tile_ops_need_general(ops.data() + h.op0, (size_t)h.nops);
        }
        const cudaError_t e = qk::launch_tile_batch(b->d_lprogs + launch[k].first, b->d_lfirst + launch[k].second, np,
                                                    ctas[k], b->d_lops, b->d_llg, b->d_llin, general, b->stream);
        if (e != cudaSuccess) return bfail(b, QK_ECUDA, "batch: tile launch failed: %s", cudaGetErrorString(e));
        ++b->large_launches;
    }
    return QK_OK;
}

}  // namespace

namespace {
// device -> host copy on the batch's stream, complete on return
bool read_back(qk_batch *b, void *dst, const void *src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, b->stream) == cudaSuccess &&
           cudaStreamSynchronize(b->stream) == cudaSuccess;
}
}  // namespace

extern "C" {

qk_status qk_batch_create(qk_batch **out, void *cuda_stream) {
    if (!out) return QK_EINVAL;
    *out = nullptr;
    qk_batch *b = new (std::nothrow) qk_batch();
    if (!b) return QK_ENOMEM;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return QK_ECUDA;
    }
    b->device = dev;
    b->pool_held = qk::pool_acquire(dev) != nullptr;
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return QK_ECUDA;
        }
        b->own_stream = true;
    }
    if (cudaEventCreate(&b->done) != cudaSuccess || cudaEventCreate(&b->start) != cudaSuccess) {
        qk_batch_destroy(b);
        return QK_ECUDA;
    }
    *out = b;
    return QK_OK;
}

qk_status qk_batch_destroy(qk_batch *b) {
    if (!b) return QK_EINVAL;
    if (b->stream) {
        void *bufs[] = {b->d_ops, b->d_circs, b->d_states, b->d_cbits, b->d_lstates, b->d_lprogs,
                        b->d_lfirst, b->d_loffs, b->d_lops, b->d_llg, b->d_llin};
        for (void *q : bufs)
            if (q) cudaFreeAsync(q, b->stream);
        cudaStreamSynchronize(b->stream);
    }
    if (b->pool_held) qk::pool_release(b->device);   // after its blocks went back to the pool
    if (b->h_stage) cudaFreeHost(b->h_stage);
    if (b->done) cudaEventDestroy(b->done);
    if (b->start) cudaEventDestroy(b->start);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return QK_OK;
}

qk_status qk_batch_clear(qk_batch *b) {
    if (!b) return QK_EINVAL;
    // the previous run may still read the staging buffer and device program
    if (cudaEventSynchronize(b->done) != cudaSuccess) return bfail(b, QK_ECUDA, "batch: event wait failed");
    b->ops.clear();
    b->circs.clear();
    b->total_amps = 0;
    b->total_cb = 0;
    b->max_n = 0;
    b->large.clear();
    b->large_of.clear();
    b->large_amps = 0;
    return QK_OK;
}

qk_status qk_batch_add_circuit(qk_batch *b, int n, int ncbits, int *index) {
    if (!b) return QK_EINVAL;
    if (n < 1 || n > qk::kBMaxLargeQubits)
        return bfail(b, QK_EINVAL, "batch: circuits take 1..%d qubits", qk::kBMaxLargeQubits);
    if (ncbits < 0 || ncbits > qk::kBMaxCbits) return bfail(b, QK_EINVAL, "batch: at most %d cbits", qk::kBMaxCbits);
    qk::BCirc c{};
    c.op_begin = c.op_end = (uint32_t)b->ops.size();
    c.n = (uint32_t)n;
    c.ncb = (uint32_t)ncbits;
    c.cb_off = b->total_cb;
    b->total_cb += (uint32_t)ncbits;
    if (index) *index = (int)b->circs.size();
    if (n > qk::kBMaxQubits) {
        qk_batch::Large L;
        L.circ = (int)b->circs.size();
        L.n = n;
        L.state_off = b->large_amps;
        b->large_amps += 1ull << n;
        c.flags |= 2u;    // a large circuit: state in the large pool, no BOps
        b->large_of.push_back((int)b->large.size());
        b->large.push_back(std::move(L));
    } else {
        c.state_off = b->total_amps;
        b->total_amps += 1ull << n;
        b->max_n = std::max(b->max_n, n);
        b->large_of.push_back(-1);
    }
    b->circs.push_back(c);
    return QK_OK;
}

qk_status qk_batch_apply_gate(qk_batch *b, int gate_id, const int *targets, int nt, const int *controls, int nc,
                              const int *cond_cbits, int ncc, const double *params, int np) {
    if (!b) return QK_EINVAL;
    qk::BCirc *c;
    if (!cur_circuit(b, &c)) return bfail(b, QK_ESTATE, "batch: add a circuit first");
    const int n = (int)c->n;
    int ntg = 0;
    if (!qk::builtin_arity(gate_id, params, np, ntg) || nt != ntg || ntg != 1)
        return bfail(b, QK_EINVAL, "batch: gate %d is not a 1-target built-in with these params", gate_id);
    if (!distinct(targets, nt, n) || nc < 0 || nc > 16 || (nc > 0 && !distinct(controls, nc, n)))
        return bfail(b, QK_EINVAL, "batch: bad qubit lists");
    uint32_t cmask = 0;
    for (int k = 0; k < nc; ++k) {
        if (controls[k] == targets[0]) return bfail(b, QK_EINVAL, "batch: control equals target");
        cmask |= 1u << controls[k];
    }
    const int q = targets[0];
    if (c->flags & 2u) {  // large circuit: ops for the tile planner
        if (ncc != 0 || nc > 1)
            return bfail(b, QK_EINVAL, "batch: circuits above %d qubits take gates with at most one control and no "
                                       "classical condition", qk::kBMaxQubits);
        // kept as a list entry; the planning threads form its matrix (append_fused)
        qk_gate_op g;
        std::memset(&g, 0, sizeof g);
        g.gate_id = gate_id;
        g.target = q;
        g.nc = nc;
        if (nc) g.controls[0] = controls[0];
        g.np = np;
        for (int k = 0; k < np; ++k) g.params[k] = params[k];
        b->large[b->large_of.back()].gates.push_back(g);
        return QK_OK;
    }
    qk::BOp op;
    std::memset(&op, 0, sizeof op);
    if (!fill_cond(op, *c, cond_cbits, ncc)) return bfail(b, QK_EINVAL, "batch: bad classical condition");
    // a gate that is never diagonal (X, Y, H, U3 with theta != 0) is kept as its id
    // and angles; qk_batch_run forms the matrices on the host's cores
    if (gate_id == QK_GATE_X || gate_id == QK_GATE_Y || gate_id == QK_GATE_H ||
        (gate_id == QK_GATE_U3 && params[0] != 0.0)) {
        op.kind = qk::B_RAW;
        op.q = (uint8_t)q;
        op.cmask = cmask;
        op.raw.id = gate_id;
        op.raw.np = np;
        for (int k = 0; k < np; ++k) op.raw.p[k] = params[k];
        b->ops.push_back(op);
        c->op_end = (uint32_t)b->ops.size();
        return QK_OK;
    }
    qk::cd m[4];
    qk::builtin_matrix(gate_id, params, np, m, ntg);   // valid: checked above
    if (m[1] == 0.0 && m[2] == 0.0) {  // diagonal: one phase op per entry that is not 1
        for (int e = 0; e < 2; ++e) {
            const qk::cd f = e ? m[3] : m[0];
            if (f == 1.0) continue;
            qk::BOp p = op;
            p.kind = qk::B_PHASE;
            p.cmask = cmask | (1u << q);
            p.val = cmask | (e ? (1u << q) : 0u);
            p.ph.re = (float)f.real();
            p.ph.im = (float)f.imag();
            b->ops.push_back(p);
        }
    } else {
        op.kind = qk::B_U2;
        op.q = (uint8_t)q;
        op.cmask = cmask;
        for (int e = 0; e < 4; ++e) {
            op.m[2 * e] = (float)m[e].real();
            op.m[2 * e + 1] = (float)m[e].imag();
        }
        b->ops.push_back(op);
    }
    c->op_end = (uint32_t)b->ops.size();
    return QK_OK;
}

qk_status qk_batch_apply_gates(qk_batch *b, const qk_gate_op *ops, int count) {
    if (!b) return QK_EINVAL;
    if (count < 0 || (count > 0 && !ops)) return bfail(b, QK_EINVAL, "batch: bad gate list");
    if (!b->large_of.empty() && b->large_of.back() >= 0) {
        auto &G = b->large[b->large_of.back()].gates;
        G.reserve(G.size() + (size_t)count);
    }
    for (int i = 0; i < count; ++i) {
        const qk_gate_op &g = ops[i];
        if (g.nc < 0 || g.nc > 4 || g.ncc < 0 || g.ncc > 4 || g.np < 0 || g.np > 3)
            return bfail(b, QK_EINVAL, "batch: gate list entry %d has bad counts", i);
        const qk_status st =
            qk_batch_apply_gate(b, g.gate_id, &g.target, 1, g.controls, g.nc, g.cond, g.ncc, g.params, g.np);
        if (st != QK_OK) {
            const std::string msg = b->err;
            return bfail(b, st, "batch: gate list entry %d: %s", i, msg.c_str());
        }
    }
    return QK_OK;
}

qk_status qk_batch_apply_mulmod(qk_batch *b, const int *targets, int w, const int *controls, int nc, uint64_t cc,
                                uint64_t N) {
    if (!b) return QK_EINVAL;
    qk::BCirc *c;
    if (!cur_circuit(b, &c)) return bfail(b, QK_ESTATE, "batch: add a circuit first");
    const int n = (int)c->n;
    if (c->flags & 2u) return bfail(b, QK_EINVAL, "batch: circuits above %d qubits take unitary gates only", qk::kBMaxQubits);
    if (w < 1 || w > 16 || !distinct(targets, w, n) || nc < 0 || (nc > 0 && !distinct(controls, nc, n)))
        return bfail(b, QK_EINVAL, "batch: bad mul-mod register or controls");
    if (N < 2 || N > (1ull << w) || cc >= N) return bfail(b, QK_EINVAL, "batch: need 2 <= N <= 2^w and c < N");
    bool ok = false;
    const uint64_t inv = qk::modinv(cc, N, ok);
    if (!ok) return bfail(b, QK_ENOTBIJECTIVE, "batch: gcd(c, N) != 1");
    qk::BOp op;
    std::memset(&op, 0, sizeof op);
    op.kind = qk::B_MULMOD;
    op.w = (uint8_t)w;
    for (int k = 0; k < w; ++k) op.mm.rpos[k] = (uint8_t)targets[k];
    for (int k = 0; k < nc; ++k) {
        for (int t = 0; t < w; ++t)
            if (controls[k] == targets[t]) return bfail(b, QK_EINVAL, "batch: control inside the register");
        op.cmask |= 1u << controls[k];
    }
    op.mm.N = (uint32_t)N;
    op.mm.cinv = (uint32_t)inv;
    c->flags |= 1u;
    b->ops.push_back(op);
    c->op_end = (uint32_t)b->ops.size();
    return QK_OK;
}

qk_status qk_batch_measure(qk_batch *b, const int *qubits, int nq, const double *uniforms, const int *dest) {
    if (!b) return QK_EINVAL;
    qk::BCirc *c;
    if (!cur_circuit(b, &c)) return bfail(b, QK_ESTATE, "batch: add a circuit first");
    if (c->flags & 2u) return bfail(b, QK_EINVAL, "batch: circuits above %d qubits take unitary gates only", qk::kBMaxQubits);
    if (nq < 1 || !distinct(qubits, nq, (int)c->n) || !uniforms) return bfail(b, QK_EINVAL, "batch: bad qubit list");
    for (int k = 0; k < nq; ++k) {
        if (!(uniforms[k] >= 0.0 && uniforms[k] < 1.0)) return bfail(b, QK_EINVAL, "batch: uniform not in [0, 1)");
        if (dest && (dest[k] < 0 || dest[k] >= (int)c->ncb)) return bfail(b, QK_EINVAL, "batch: bad destination cbit");
        qk::BOp op;
        std::memset(&op, 0, sizeof op);
        op.kind = qk::B_MEASURE;
        op.q = (uint8_t)qubits[k];
        op.ms.u = uniforms[k];
        op.ms.dest = dest ? dest[k] : -1;
        b->ops.push_back(op);
    }
    c->op_end = (uint32_t)b->ops.size();
    return QK_OK;
}

qk_status qk_batch_run(qk_batch *b, int store_states) {
    if (!b) return QK_EINVAL;
    if (b->circs.empty()) return QK_OK;
    b->store_state = store_states != 0;
    b->start_recorded = false;
    b->plan_ms = 0.0;
    b->large_launches = 0;
    // large circuits first: their planning is host work, after which the start
    // event is recorded and everything else is enqueued back to back
    if (!b->large.empty()) {
        const qk_status ls = run_large(b);
        if (ls != QK_OK) return ls;
    } else {
        if (cudaEventRecord(b->start, b->stream) != cudaSuccess) return bfail(b, QK_ECUDA, "batch: event record failed");
        b->start_recorded = true;
    }
    qk_status s;
    if ((s = grow(b, &b->d_ops, &b->cap_ops, std::max<size_t>(1, b->ops.size()))) != QK_OK) return s;
    if ((s = grow(b, &b->d_circs, &b->cap_circs, std::max<size_t>(1, b->circs.size()))) != QK_OK) return s;
    if (b->store_state && (s = grow(b, &b->d_states, &b->cap_states, b->total_amps)) != QK_OK) return s;
    if ((s = grow(b, &b->d_cbits, &b->cap_cbits, std::max<size_t>(1, b->total_cb))) != QK_OK) return s;
    // circuits of at most 13 qubits, sorted by size: one launch per qubit count (and
    // per need of the second state buffer, which only mul-mod gathers use), each
    // sized to its shared memory (small circuits then share an SM)
    std::vector<qk::BCirc> sorted;
    for (const auto &c : b->circs)
        if (!(c.flags & 2u)) sorted.push_back(c);
    std::stable_sort(sorted.begin(), sorted.end(), [](const qk::BCirc &x, const qk::BCirc &y) {
        return x.n != y.n ? x.n < y.n : (x.flags & 1u) < (y.flags & 1u);
    });
    form_raw_ops(b->ops);
    // stage the program in pinned memory so that the copies are truly asynchronous
    const size_t ob = sizeof(qk::BOp) * b->ops.size(), cb = sizeof(qk::BCirc) * sorted.size();
    if (ob + cb > 0 && ob + cb > b->cap_stage) {
        if (b->h_stage) cudaFreeHost(b->h_stage);
        b->h_stage = nullptr;
        b->cap_stage = 0;
        if (cudaMallocHost(&b->h_stage, (ob + cb) * 2) != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, QK_ENOMEM, "batch: cannot allocate pinned staging");
        }
        b->cap_stage = (ob + cb) * 2;
    }
    if (ob + cb > 0) {
        std::memcpy(b->h_stage, b->ops.data(), ob);
        std::memcpy((char *)b->h_stage + ob, sorted.data(), cb);
        if (cudaMemcpyAsync(b->d_ops, b->h_stage, ob, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
            cudaMemcpyAsync(b->d_circs, (char *)b->h_stage + ob, cb, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
            return bfail(b, QK_ECUDA, "batch: upload failed");
    }
    const size_t max_smem = sizeof(float2) * 2 * ((size_t)1 << b->max_n);
    if (!sorted.empty() && max_smem > 48 * 1024 &&
        cudaFuncSetAttribute(qk::k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem) != cudaSuccess)
        return bfail(b, QK_ECUDA, "batch: shared memory attribute failed");
    for (size_t i = 0; i < sorted.size();) {
        size_t j = i;
        while (j < sorted.size() && sorted[j].n == sorted[i].n && (sorted[j].flags & 1u) == (sorted[i].flags & 1u))
            ++j;
        const size_t smem = sizeof(float2) * ((sorted[i].flags & 1u) ? 2 : 1) * ((size_t)1 << sorted[i].n);
        qk::k_batch<<<(unsigned)(j - i), qk::kBThreads, smem, b->stream>>>(b->d_circs + i, b->d_ops, b->d_states,
                                                                          b->d_cbits, b->store_state ? 1 : 0);
        if (cudaGetLastError() != cudaSuccess) return bfail(b, QK_ECUDA, "batch: launch failed");
        i = j;
    }
    if (cudaEventRecord(b->done, b->stream) != cudaSuccess) return bfail(b, QK_ECUDA, "batch: event record failed");
    return QK_OK;
}

qk_status qk_batch_stats(qk_batch *b, double *plan_ms, int *tile_launches, double *device_ms) {
    if (!b) return QK_EINVAL;
    if (plan_ms) *plan_ms = b->plan_ms;
    if (tile_launches) *tile_launches = b->large_launches;
    if (device_ms) {
        *device_ms = 0.0;
        if (b->start_recorded) {
            float ms = 0.f;
            if (cudaEventSynchronize(b->done) != cudaSuccess || cudaEventElapsedTime(&ms, b->start, b->done) != cudaSuccess)
                return bfail(b, QK_ECUDA, "batch: event timing failed");
            *device_ms = ms;
        }
    }
    return QK_OK;
}

int qk_batch_done(qk_batch *b) {
    if (!b) return -1;
    const cudaError_t e = cudaEventQuery(b->done);
    if (e == cudaSuccess) return 1;
    if (e == cudaErrorNotReady) {
        cudaGetLastError();
        return 0;
    }
    return -1;
}

qk_status qk_batch_read(qk_batch *b, int circuit, uint8_t *cbits, int ncb, void *state, size_t bytes) {
    if (!b) return QK_EINVAL;
    if (circuit < 0 || circuit >= (int)b->circs.size()) return bfail(b, QK_EINVAL, "batch: bad circuit index");
    const qk::BCirc &c = b->circs[circuit];
    if (ncb < 0 || ncb > (int)c.ncb || (ncb > 0 && !cbits)) return bfail(b, QK_EINVAL, "batch: bad cbit count");
    const bool large = (c.flags & 2u) != 0;
    if (state && ((!large && !b->store_state) || bytes != sizeof(float2) << c.n))
        return bfail(b, QK_EINVAL, "batch: state not stored or wrong size (%zu bytes expected)", sizeof(float2) << c.n);
    if (cudaEventSynchronize(b->done) != cudaSuccess) return bfail(b, QK_ECUDA, "batch: event wait failed");
    // reads on the batch's own stream (its run is complete: the event above)
    if (ncb > 0 && !read_back(b, cbits, b->d_cbits + c.cb_off, ncb))
        return bfail(b, QK_ECUDA, "batch: cbit copy failed");
    const float2 *src = large ? b->d_lstates + b->large[b->large_of[circuit]].state_off : b->d_states + c.state_off;
    if (state && !read_back(b, state, src, bytes)) return bfail(b, QK_ECUDA, "batch: state copy failed");
    return QK_OK;
}

qk_status qk_batch_read_all_cbits(qk_batch *b, uint8_t *out, size_t n) {
    if (!b) return QK_EINVAL;
    if (n != b->total_cb || (n > 0 && !out)) return bfail(b, QK_EINVAL, "batch: need %u cbit bytes", b->total_cb);
    if (cudaEventSynchronize(b->done) != cudaSuccess) return bfail(b, QK_ECUDA, "batch: event wait failed");
    if (n > 0 && !read_back(b, out, b->d_cbits, n)) return bfail(b, QK_ECUDA, "batch: cbit copy failed");
    return QK_OK;
}

int qk_batch_num_circuits(const qk_batch *b) { return b ? (int)b->circs.size() : -1; }

const char *qk_batch_last_error(const qk_batch *b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
