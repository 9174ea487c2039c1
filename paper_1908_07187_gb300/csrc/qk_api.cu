// Host side of libqk: the C ABI of include/qk.h, gate decomposition into
// device launches, qubit relabelling (SWAP), measurement sequencing and the
// fused-mode queue.  All arithmetic on amplitudes happens in the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "qk.h"
#include "qk_kernels.cuh"
#include "qk_host.h"
#include "qk_plan.h"

using cd = std::complex<double>;

namespace qk {
namespace {
constexpr int kPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kPoolDevices] = {};
int g_pool_users[kPoolDevices] = {};
}  // namespace

cudaMemPool_t pool_acquire(int device) {
    if (device < 0 || device >= kPoolDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[device]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;   // keep freed blocks for reuse
        if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            cudaGetLastError();
            cudaMemPoolDestroy(pool);
            return nullptr;
        }
        g_pool[device] = pool;
    }
    ++g_pool_users[device];
    return g_pool[device];
}

void pool_release(int device) {
    if (device < 0 || device >= kPoolDevices) return;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[device] || g_pool_users[device] <= 0) return;
    if (--g_pool_users[device] == 0) cudaMemPoolTrimTo(g_pool[device], 0);   // the last holder: give it all back
}

cudaError_t pool_malloc(void **p, size_t bytes, int device, cudaStream_t s) {
    cudaMemPool_t pool = nullptr;
    if (device >= 0 && device < kPoolDevices) {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        pool = g_pool[device];
    }
    if (pool) return cudaMallocFromPoolAsync(p, bytes, pool, s);
    return cudaMallocAsync(p, bytes, s);
}
}  // namespace qk

namespace {

struct GateDef {
    int kind = 0;                 // 0 = matrix, 1 = mul-mod, 2 = table
    int k = 0;                    // matrix qubits, or register width w
    std::vector<cd> m;            // FP64 master matrix (row-major)
    bool diagonal = false;
    void *d_mat = nullptr;        // working-precision copy on the device
    uint64_t c = 0, N = 0, cinv = 0;
    uint32_t *d_finv = nullptr;
    // 5-qubit gates on the tensor cores: split real embeddings per target order
    std::vector<std::pair<uint32_t, float *>> tc_cache;
};

struct ProfRec {
    int cls;
    cudaEvent_t a, b;
    double bytes;
};

constexpr int kMeasBlocksPerSM = 8;   // measurement reductions: enough loads in flight for HBM

}  // namespace

struct qk_ctx {
    qk_precision prec = QK_C64;
    size_t amp = 8;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool pool_held = false;   // holds the library's memory pool of its device
    int device = 0;
    int sms = 148;
    qk_options opt{};

    int n = 0;
    void *d_state = nullptr;
    void *d_scratch = nullptr;
    size_t state_bytes = 0, scratch_bytes = 0;

    int ncb = 0, cb_cap = 0;
    uint8_t *d_cbits = nullptr;

    double *d_partials = nullptr;
    int *d_err = nullptr;          // set by a kernel whose bounded wait gave up
    unsigned *d_counter = nullptr; // reduction ticket (zero between launches)
    int meas_blocks = 0;
    qk::MeasSlot *d_slots = nullptr;
    int slot_cap = 0;

    std::vector<int> l2p;          // logical -> physical qubit
    std::vector<GateDef> gates;
    void *d_swap_mat = nullptr;    // SWAP as a 4x4 matrix, for controlled SWAPs

    std::vector<qk::FusedOp> pending;   // fused-mode queue (physical qubits)
    qk::TilePlanner *planner = nullptr;

    uint64_t launches = 0, passes_x1000 = 0;
    double alg_bytes = 0.0;
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
    uint64_t prof_launches[QK_NUM_LAUNCH_CLASSES] = {};
    double prof_ms[QK_NUM_LAUNCH_CLASSES] = {};
    double prof_bytes[QK_NUM_LAUNCH_CLASSES] = {};

    bool capturing = false;       // the stream is being captured into a CUDA graph
    void *cap_state0 = nullptr;   // state buffer when the capture began

    std::string err;
};

struct qk_graph {
    qk_ctx *ctx;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace {

qk_status fail(qk_ctx *c, qk_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

#define CUDA_TRY(ctx, call)                                                                      \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail((ctx), QK_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
    } while (0)

size_t full_pass_bytes(const qk_ctx *c) { return (size_t)2 * c->amp << c->n; }


// Device memory is stream-ordered on the context's stream (from the library's
// pool, freed with cudaFreeAsync): freeing a finished context does not
// synchronise the device, so other contexts' work keeps running (the serving
// loop relies on this).
cudaError_t dalloc(qk_ctx *c, void **p, size_t bytes) { return qk::pool_malloc(p, bytes, c->device, c->stream); }
void dfree(qk_ctx *c, void *p) {
    if (p) cudaFreeAsync(p, c->stream);
}
// host -> device copy of a small pageable buffer, complete before return
cudaError_t upload(qk_ctx *c, void *dst, const void *src, size_t bytes) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream);
    return e == cudaSuccess ? cudaStreamSynchronize(c->stream) : e;
}

cudaEvent_t get_event(qk_ctx *c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket a launch with CUDA events when profiling; count it either way.
struct LaunchScope {
    qk_ctx *c;
    int cls;
    double bytes;
    cudaEvent_t a = nullptr;
    LaunchScope(qk_ctx *c_, int cls_, double bytes_) : c(c_), cls(cls_), bytes(bytes_) {
        if (c->opt.profile && !c->capturing) {
            a = get_event(c);
            cudaEventRecord(a, c->stream);
        }
    }
    ~LaunchScope() {
        c->launches++;
        c->alg_bytes += bytes;
        const double fp = (double)full_pass_bytes(c);
        if (fp > 0) c->passes_x1000 += (uint64_t)llround(1000.0 * bytes / fp);
        if (c->opt.profile && !c->capturing) {
            cudaEvent_t b = get_event(c);
            cudaEventRecord(b, c->stream);
            c->prof.push_back({cls, a, b, bytes});
        }
    }
};

#define NOT_WHILE_CAPTURING(c, what)                                                   \
    do {                                                                               \
        if ((c)->capturing) return fail((c), QK_ESTATE, "%s is not allowed while capturing", what); \
    } while (0)

bool valid_qubits(const qk_ctx *c, const int *q, int k) {
    if (k < 0 || (k > 0 && !q)) return false;
    for (int a = 0; a < k; ++a) {
        if (q[a] < 0 || q[a] >= c->n) return false;
        for (int b = 0; b < a; ++b)
            if (q[a] == q[b]) return false;
    }
    return true;
}

bool fill_cond(qk_ctx *c, qk::Cond &cond, const int *cb, int ncc) {
    if (ncc < 0 || ncc > qk::kMaxCond || (ncc > 0 && !cb)) return false;
    cond.n = ncc;
    for (int a = 0; a < ncc; ++a) {
        if (cb[a] < 0 || cb[a] >= c->ncb) return false;
        cond.idx[a] = cb[a];
    }
    return true;
}

void set_positions(qk::Positions &p, std::vector<int> v) {
    std::sort(v.begin(), v.end());
    p.n = (int)v.size();
    for (int a = 0; a < p.n; ++a) p.pos[a] = v[a];
}

// Upload a matrix in the working precision.
qk_status upload_matrix(qk_ctx *c, const std::vector<cd> &m, void **dptr) {
    const size_t cnt = m.size();
    std::vector<unsigned char> host(cnt * c->amp);
    for (size_t i = 0; i < cnt; ++i) {
        if (c->prec == QK_C64) {
            float v[2] = {(float)m[i].real(), (float)m[i].imag()};
            memcpy(&host[i * 8], v, 8);
        } else {
            double v[2] = {m[i].real(), m[i].imag()};
            memcpy(&host[i * 16], v, 16);
        }
    }
    CUDA_TRY(c, dalloc(c, dptr, host.size()));
    CUDA_TRY(c, upload(c, *dptr, host.data(), host.size()));
    return QK_OK;
}

// ---------------------------------------------------------------------------
// plain execution of one fused-queue op
// ---------------------------------------------------------------------------
qk_status run_op_plain(qk_ctx *c, const qk::FusedOp &op) {
    const int n = c->n;
    if (op.kind == qk::FusedOp::U2) {
        qk::U2Args a{};
        for (int i = 0; i < 4; ++i) {
            a.m[2 * i] = op.m[i].real();
            a.m[2 * i + 1] = op.m[i].imag();
        }
        a.cmask = op.cmask;
        a.q = op.q;
        std::vector<int> pos{op.q};
        for (int b = 0; b < n; ++b)
            if ((op.cmask >> b) & 1) pos.push_back(b);
        set_positions(a.ins, pos);
        a.n_units = 1ull << (n - (int)pos.size());
        a.cond = op.cond;
        LaunchScope ls(c, 1, (double)2 * c->amp * (double)(1ull << (n - (int)pos.size() + 1)));
        CUDA_TRY(c, qk::launch_u2((int)c->prec, c->d_state, a, c->d_cbits, n, c->sms, c->stream));
    } else if (op.kind == qk::FusedOp::PHASE) {
        qk::PhaseArgs a{};
        a.f_re = op.f.real();
        a.f_im = op.f.imag();
        a.mask = op.mask;
        a.val = op.val;
        std::vector<int> pos;
        for (int b = 0; b < n; ++b)
            if ((op.mask >> b) & 1) pos.push_back(b);
        set_positions(a.ins, pos);
        a.n_units = 1ull << (n - (int)pos.size());
        a.cond = op.cond;
        a.n_rphase = 0;
        LaunchScope ls(c, 2, (double)2 * c->amp * (double)a.n_units);
        CUDA_TRY(c, qk::launch_phase((int)c->prec, c->d_state, a, c->d_cbits, c->sms, c->stream));
    } else {
        return fail(c, QK_EINVAL, "internal: unknown queued op kind");
    }
    return QK_OK;
}

qk_status flush(qk_ctx *c) {
    if (c->pending.empty()) return QK_OK;
    qk_status st = QK_OK;
    if (c->opt.exec_mode == QK_EXEC_FUSED && c->planner) {
        st = qk::run_fused(c->planner, c, c->pending);
    } else {
        for (const auto &op : c->pending) {
            st = run_op_plain(c, op);
            if (st != QK_OK) break;
        }
    }
    c->pending.clear();
    return st;
}

qk_status enqueue(qk_ctx *c, const qk::FusedOp &op) {
    if (c->opt.exec_mode == QK_EXEC_PLAIN) return run_op_plain(c, op);
    c->pending.push_back(op);
    if ((int)c->pending.size() >= c->opt.max_pending) return flush(c);
    return QK_OK;
}

// Queue a (controlled) 1-qubit matrix on physical qubit q.
qk_status apply_1q(qk_ctx *c, const cd m[4], int q, uint64_t cmask, const qk::Cond &cond) {
    const uint64_t tb = 1ull << q;
    if (m[1] == 0.0 && m[2] == 0.0) {
        // diagonal: one phase op per entry that differs from 1
        if (m[0] != 1.0) {
            qk::FusedOp op;
            op.kind = qk::FusedOp::PHASE;
            op.mask = cmask | tb;
            op.val = cmask;
            op.f = m[0];
            op.cond = cond;
            qk_status s = enqueue(c, op);
            if (s != QK_OK) return s;
        }
        if (m[3] != 1.0) {
            qk::FusedOp op;
            op.kind = qk::FusedOp::PHASE;
            op.mask = cmask | tb;
            op.val = cmask | tb;
            op.f = m[3];
            op.cond = cond;
            return enqueue(c, op);
        }
        return QK_OK;
    }
    qk::FusedOp op;
    op.kind = qk::FusedOp::U2;
    op.q = q;
    op.cmask = cmask;
    for (int i = 0; i < 4; ++i) op.m[i] = m[i];
    op.cond = cond;
    return enqueue(c, op);
}

qk_status ensure_scratch(qk_ctx *c) {
    if (c->d_scratch && c->scratch_bytes == c->state_bytes) return QK_OK;
    if (c->capturing) return fail(c, QK_ESTATE, "a gather buffer would be allocated during capture");
    dfree(c, c->d_scratch);
    c->d_scratch = nullptr;
    c->scratch_bytes = 0;
    if (c->opt.hbm_budget_bytes && 2 * c->state_bytes > c->opt.hbm_budget_bytes)
        return fail(c, QK_EBUDGET, "permutation scratch (%zu bytes) exceeds the HBM budget", c->state_bytes);
    if (dalloc(c, &c->d_scratch, c->state_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, QK_ENOMEM, "cannot allocate %zu bytes of permutation scratch", c->state_bytes);
    }
    c->scratch_bytes = c->state_bytes;
    return QK_OK;
}

// Physically reorder the state so that logical qubit q is physical bit q.
qk_status canonicalize(qk_ctx *c) {
    bool ident = true;
    for (int q = 0; q < c->n; ++q) ident = ident && c->l2p[q] == q;
    if (ident) return QK_OK;
    qk_status s = ensure_scratch(c);
    if (s != QK_OK) return s;
    qk::RelabelArgs a{};
    a.n = c->n;
    for (int q = 0; q < c->n; ++q) a.phys_of[q] = c->l2p[q];
    a.n_amps = 1ull << c->n;
    {
        LaunchScope ls(c, 6, (double)full_pass_bytes(c));
        CUDA_TRY(c, qk::launch_relabel((int)c->prec, c->d_state, c->d_scratch, a, c->sms, c->stream));
    }
    std::swap(c->d_state, c->d_scratch);
    for (int q = 0; q < c->n; ++q) c->l2p[q] = q;
    return QK_OK;
}

qk_status ensure_slots(qk_ctx *c, int nq) {
    if (nq <= c->slot_cap) return QK_OK;
    if (c->capturing) return fail(c, QK_ESTATE, "measurement slots would be allocated during capture");
    dfree(c, c->d_slots);
    c->d_slots = nullptr;
    int cap = std::max(nq, 64);
    CUDA_TRY(c, dalloc(c, (void **)&c->d_slots, sizeof(qk::MeasSlot) * cap));
    c->slot_cap = cap;
    return QK_OK;
}

// Move the logical qubits targets[0..k-1] onto physical qubits 0..k-1 with one
// relabelling gather: each target above k-1 trades places with a non-target
// qubit on a low position; the logical -> physical map records the move.
qk_status move_to_low(qk_ctx *c, const int *targets, int k) {
    const int n = c->n;
    std::vector<int> inv(n), newp(c->l2p);
    for (int q = 0; q < n; ++q) inv[c->l2p[q]] = q;
    std::vector<char> is_target(n, 0);
    for (int a = 0; a < k; ++a) is_target[targets[a]] = 1;
    std::vector<int> free_low;
    for (int p = 0; p < k; ++p)
        if (!is_target[inv[p]]) free_low.push_back(p);
    size_t fi = 0;
    bool moved = false;
    for (int a = 0; a < k; ++a) {
        const int p = c->l2p[targets[a]];
        if (p < k) continue;
        const int f = free_low[fi++];
        newp[targets[a]] = f;
        newp[inv[f]] = p;
        moved = true;
    }
    if (!moved) return QK_OK;
    qk_status s = ensure_scratch(c);
    if (s != QK_OK) return s;
    std::vector<int> newinv(n);
    for (int q = 0; q < n; ++q) newinv[newp[q]] = q;
    qk::RelabelArgs a{};
    a.n = n;
    for (int p2 = 0; p2 < n; ++p2) a.phys_of[p2] = c->l2p[newinv[p2]];   // new bit p2 <- old bit
    a.n_amps = 1ull << n;
    {
        LaunchScope ls(c, 6, (double)full_pass_bytes(c));
        CUDA_TRY(c, qk::launch_relabel((int)c->prec, c->d_state, c->d_scratch, a, c->sms, c->stream));
    }
    std::swap(c->d_state, c->d_scratch);
    c->l2p = newp;
    return QK_OK;
}

// Dense 5-qubit gate on physical qubits 0..4 via the tensor-core kernel.  The
// real embedding of U, with rows and columns permuted to the physical order of
// the targets, is split into TF32 high and low parts once per target order.
// A k-qubit gate (k = 3, 4) is the 5-qubit block U (x) I on its targets and the
// other low physical qubits: entries whose spectator bits differ are zero.
qk_status apply_block_tc(qk_ctx *c, int gate_id, const int *targets, uint32_t key) {
    GateDef &g = c->gates[gate_id];
    const int k = g.k;
    float *dev = nullptr;
    for (auto &e : g.tc_cache)
        if (e.first == key) dev = e.second;
    if (!dev) {
        if (c->capturing) return fail(c, QK_ESTATE, "tensor-core matrices would be allocated during capture");
        int pa[5];
        int tmask = 0;
        for (int a = 0; a < k; ++a) {
            pa[a] = c->l2p[targets[a]];
            tmask |= 1 << pa[a];
        }
        auto value = [&](int x) {  // gate register value of physical low-bit index x
            int v = 0;
            for (int a = 0; a < k; ++a) v |= ((x >> pa[a]) & 1) << (k - 1 - a);
            return v;
        };
        const size_t d = (size_t)1 << k;
        std::vector<float> bh(64 * 64), bl(64 * 64);
        for (int r = 0; r < 32; ++r)
            for (int x = 0; x < 32; ++x) {
                const cd u = ((r & ~tmask) == (x & ~tmask)) ? g.m[(size_t)value(r) * d + value(x)] : cd(0.0);
                const float re = (float)u.real(), im = (float)u.imag();
                const float vals[4] = {re, -im, im, re};          // (2r,2x) (2r,2x+1) (2r+1,2x) (2r+1,2x+1)
                const int idx[4] = {(2 * r) * 64 + 2 * x, (2 * r) * 64 + 2 * x + 1, (2 * r + 1) * 64 + 2 * x,
                                    (2 * r + 1) * 64 + 2 * x + 1};
                for (int q = 0; q < 4; ++q) {
                    uint32_t bits;
                    std::memcpy(&bits, &vals[q], 4);
                    bits &= 0xFFFFE000u;
                    float hi;
                    std::memcpy(&hi, &bits, 4);
                    bh[idx[q]] = hi;
                    bl[idx[q]] = vals[q] - hi;
                }
            }
        CUDA_TRY(c, dalloc(c, (void **)&dev, sizeof(float) * 2 * 64 * 64));
        CUDA_TRY(c, upload(c, dev, bh.data(), sizeof(float) * 64 * 64));
        CUDA_TRY(c, upload(c, dev + 64 * 64, bl.data(), sizeof(float) * 64 * 64));
        g.tc_cache.push_back({key, dev});
    }
    LaunchScope ls(c, 3, (double)full_pass_bytes(c));
    CUDA_TRY(c, qk::launch_block_tc(c->d_state, c->n, dev, dev + 64 * 64, c->d_err, c->sms, c->stream));
    return QK_OK;
}

}  // namespace

// ===========================================================================
// fused-mode hooks used by the planner (qk_plan.cu)
// ===========================================================================
namespace qk {
void *ctx_state(qk_ctx *c) { return c->d_state; }
int ctx_n(qk_ctx *c) { return c->n; }
int ctx_prec(qk_ctx *c) { return (int)c->prec; }
int ctx_sms(qk_ctx *c) { return c->sms; }
int ctx_tile_qubits(qk_ctx *c) { return c->opt.tile_qubits; }
cudaStream_t ctx_stream(qk_ctx *c) { return c->stream; }
const uint8_t *ctx_cbits(qk_ctx *c) { return c->d_cbits; }
qk_status ctx_run_plain(qk_ctx *c, const FusedOp &op) { return run_op_plain(c, op); }
qk_status ctx_fail(qk_ctx *c, qk_status s, const char *msg) { return fail(c, s, "%s", msg); }
void ctx_launch_begin(qk_ctx *c, int cls, double bytes, void **token) {
    *token = new LaunchScope(c, cls, bytes);
}
void ctx_launch_end(void *token) { delete static_cast<LaunchScope *>(token); }
}  // namespace qk

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *qk_status_str(qk_status s) {
    switch (s) {
        case QK_OK: return "QK_OK";
        case QK_EINVAL: return "QK_EINVAL";
        case QK_ENOMEM: return "QK_ENOMEM";
        case QK_EBUDGET: return "QK_EBUDGET";
        case QK_ENOTBIJECTIVE: return "QK_ENOTBIJECTIVE";
        case QK_ENOTUNITARY: return "QK_ENOTUNITARY";
        case QK_ECUDA: return "QK_ECUDA";
        case QK_ETIMEOUT: return "QK_ETIMEOUT";
        case QK_ESTATE: return "QK_ESTATE";
    }
    return "unknown";
}

qk_status qk_create(qk_ctx **out, qk_precision precision, void *cuda_stream, const qk_options *opt) {
    if (!out) return QK_EINVAL;
    *out = nullptr;
    if (precision != QK_C64 && precision != QK_C128) return QK_EINVAL;
    qk_ctx *c = new (std::nothrow) qk_ctx();
    if (!c) return QK_ENOMEM;
    c->prec = precision;
    c->amp = precision == QK_C64 ? 8 : 16;
    if (opt) {
        c->opt = *opt;
        for (int r : opt->reserved)
            if (r != 0) { delete c; return QK_EINVAL; }
    } else {
        c->opt.exec_mode = QK_EXEC_FUSED;
    }
    if (c->opt.exec_mode != QK_EXEC_PLAIN && c->opt.exec_mode != QK_EXEC_FUSED) { delete c; return QK_EINVAL; }
    if (c->opt.max_pending <= 0) c->opt.max_pending = 4096;
    // the tile kernel's width is fixed: 0 (default) or that width
    if (c->opt.tile_qubits != 0 && c->opt.tile_qubits != qk::kTileQubits) { delete c; return QK_EINVAL; }
    if (c->opt.no_tensor_cores != 0 && c->opt.no_tensor_cores != 1) { delete c; return QK_EINVAL; }
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return QK_ECUDA;
    }
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return QK_ECUDA; }
        c->own_stream = true;
    }
    c->pool_held = qk::pool_acquire(c->device) != nullptr;
    c->meas_blocks = c->sms * kMeasBlocksPerSM;
    if (dalloc(c, (void **)&c->d_partials, sizeof(double) * 2 * c->meas_blocks) != cudaSuccess ||
        dalloc(c, (void **)&c->d_err, sizeof(int)) != cudaSuccess ||
        dalloc(c, (void **)&c->d_counter, sizeof(unsigned)) != cudaSuccess ||
        cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream) != cudaSuccess) {
        cudaGetLastError();
        qk_destroy(c);
        return QK_ENOMEM;
    }
    std::vector<cd> sw = {1, 0, 0, 0, 0, 0, 1, 0, 0, 1, 0, 0, 0, 0, 0, 1};
    if (upload_matrix(c, sw, &c->d_swap_mat) != QK_OK) { qk_destroy(c); return QK_ECUDA; }
    c->planner = qk::make_planner();
    *out = c;
    return QK_OK;
}

qk_status qk_destroy(qk_ctx *c) {
    if (!c) return QK_EINVAL;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto &p : c->prof) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (auto &g : c->gates) {
        dfree(c, g.d_mat);
        dfree(c, g.d_finv);
        for (auto &e : g.tc_cache) dfree(c, e.second);
    }
    dfree(c, c->d_err);
    dfree(c, c->d_counter);
    dfree(c, c->d_swap_mat);
    dfree(c, c->d_state);
    dfree(c, c->d_scratch);
    dfree(c, c->d_cbits);
    dfree(c, c->d_partials);
    dfree(c, c->d_slots);
    if (c->stream) cudaStreamSynchronize(c->stream);   // this stream only
    if (c->pool_held) qk::pool_release(c->device);     // after its blocks went back to the pool
    if (c->planner) qk::free_planner(c->planner);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return QK_OK;
}

qk_status qk_add_qubits(qk_ctx *c, int k, int *first) {
    if (!c) return QK_EINVAL;
    NOT_WHILE_CAPTURING(c, "add_qubits");
    if (k < 1 || c->n + k > QK_MAX_QUBITS) return fail(c, QK_EINVAL, "add_qubits: bad count %d (have %d)", k, c->n);
    qk_status s = flush(c);
    if (s != QK_OK) return s;
    s = canonicalize(c);
    if (s != QK_OK) return s;
    const int nn = c->n + k;
    const size_t bytes = c->amp << nn;
    if (c->opt.hbm_budget_bytes && bytes > c->opt.hbm_budget_bytes)
        return fail(c, QK_EBUDGET, "state of %d qubits (%zu bytes) exceeds the HBM budget", nn, bytes);
    void *d = nullptr;
    if (dalloc(c, &d, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, QK_ENOMEM, "cannot allocate %zu bytes for %d qubits", bytes, nn);
    }
    CUDA_TRY(c, cudaMemsetAsync(d, 0, bytes, c->stream));
    if (c->d_state) {
        CUDA_TRY(c, cudaMemcpyAsync(d, c->d_state, c->state_bytes, cudaMemcpyDeviceToDevice, c->stream));
        dfree(c, c->d_state);
    } else {
        CUDA_TRY(c, qk::launch_set_basis((int)c->prec, d, 0, c->stream));
    }
    if (c->d_scratch) {
        dfree(c, c->d_scratch);
        c->d_scratch = nullptr;
        c->scratch_bytes = 0;
    }
    if (first) *first = c->n;
    for (int q = c->n; q < nn; ++q) c->l2p.push_back(q);
    c->d_state = d;
    c->state_bytes = bytes;
    c->n = nn;
    return QK_OK;
}

qk_status qk_add_cbits(qk_ctx *c, int k, int *first) {
    if (!c) return QK_EINVAL;
    NOT_WHILE_CAPTURING(c, "add_cbits");
    if (k < 1 || c->ncb + k > (1 << 20)) return fail(c, QK_EINVAL, "add_cbits: bad count %d", k);
    if (c->ncb + k > c->cb_cap) {
        int cap = std::max(c->ncb + k, std::max(64, 2 * c->cb_cap));
        uint8_t *d = nullptr;
        CUDA_TRY(c, dalloc(c, (void **)&d, cap));
        CUDA_TRY(c, cudaMemsetAsync(d, 0, cap, c->stream));
        if (c->d_cbits) {
            CUDA_TRY(c, cudaMemcpyAsync(d, c->d_cbits, c->ncb, cudaMemcpyDeviceToDevice, c->stream));
            dfree(c, c->d_cbits);
        }
        c->d_cbits = d;
        c->cb_cap = cap;
    }
    if (first) *first = c->ncb;
    c->ncb += k;
    return QK_OK;
}

qk_status qk_define_gate_matrix(qk_ctx *c, int k, const double *u, double tol, int *gate_id) {
    if (!c) return QK_EINVAL;
    NOT_WHILE_CAPTURING(c, "define_gate_matrix");
    if (k < 1 || k > QK_MAX_MATRIX_QUBITS || !u || !gate_id || !(tol >= 0))
        return fail(c, QK_EINVAL, "define_gate_matrix: bad arguments");
    const int d = 1 << k;
    GateDef g;
    g.kind = 0;
    g.k = k;
    g.m.resize((size_t)d * d);
    for (int i = 0; i < d * d; ++i) g.m[i] = cd(u[2 * i], u[2 * i + 1]);
    double dev = 0.0;
    for (int r = 0; r < d; ++r)
        for (int cc = 0; cc < d; ++cc) {
            cd s = 0;
            for (int x = 0; x < d; ++x) s += std::conj(g.m[x * d + r]) * g.m[x * d + cc];
            dev = std::max(dev, std::abs(s - (r == cc ? 1.0 : 0.0)));
        }
    if (!(dev <= tol)) return fail(c, QK_ENOTUNITARY, "matrix is not unitary: max |U^H U - I| = %g", dev);
    g.diagonal = true;
    for (int r = 0; r < d; ++r)
        for (int cc = 0; cc < d; ++cc)
            if (r != cc && g.m[r * d + cc] != 0.0) g.diagonal = false;
    qk_status s = upload_matrix(c, g.m, &g.d_mat);
    if (s != QK_OK) return s;
    *gate_id = (int)c->gates.size();
    c->gates.push_back(std::move(g));
    return QK_OK;
}

qk_status qk_define_gate_perm_mulmod(qk_ctx *c, int w, uint64_t cc, uint64_t N, int *gate_id) {
    if (!c) return QK_EINVAL;
    NOT_WHILE_CAPTURING(c, "define_gate_perm_mulmod");
    if (w < 1 || w > QK_MAX_PERM_QUBITS || !gate_id || N < 2 || N > (1ull << w))
        return fail(c, QK_EINVAL, "define_gate_perm_mulmod: bad w=%d or N=%llu", w, (unsigned long long)N);
    if (cc >= N) return fail(c, QK_EINVAL, "define_gate_perm_mulmod: c must be < N");
    bool ok = false;
    uint64_t inv = qk::modinv(cc, N, ok);
    if (!ok) return fail(c, QK_ENOTBIJECTIVE, "x -> %llu x mod %llu is not a permutation (gcd != 1)",
                         (unsigned long long)cc, (unsigned long long)N);
    GateDef g;
    g.kind = 1;
    g.k = w;
    g.c = cc;
    g.N = N;
    g.cinv = inv;
    *gate_id = (int)c->gates.size();
    c->gates.push_back(std::move(g));
    return QK_OK;
}

qk_status qk_define_gate_perm_table(qk_ctx *c, int w, const uint64_t *f, int *gate_id) {
    if (!c) return QK_EINVAL;
    NOT_WHILE_CAPTURING(c, "define_gate_perm_table");
    if (w < 1 || w > 24 || !f || !gate_id) return fail(c, QK_EINVAL, "define_gate_perm_table: bad arguments");
    const uint64_t d = 1ull << w;
    std::vector<uint32_t> inv(d, 0xffffffffu);
    for (uint64_t x = 0; x < d; ++x) {
        if (f[x] >= d || inv[f[x]] != 0xffffffffu)
            return fail(c, QK_ENOTBIJECTIVE, "table is not a permutation (entry %llu)", (unsigned long long)x);
        inv[f[x]] = (uint32_t)x;
    }
    GateDef g;
    g.kind = 2;
    g.k = w;
    CUDA_TRY(c, dalloc(c, (void **)&g.d_finv, sizeof(uint32_t) * d));
    CUDA_TRY(c, upload(c, g.d_finv, inv.data(), sizeof(uint32_t) * d));
    *gate_id = (int)c->gates.size();
    c->gates.push_back(std::move(g));
    return QK_OK;
}

qk_status qk_apply_gate(qk_ctx *c, int gate_id, const int *targets, int nt, const int *controls, int nc,
                        const int *cond_cbits, int ncc, const double *params, int np) {
    if (!c) return QK_EINVAL;
    if (c->n == 0) return fail(c, QK_ESTATE, "apply_gate: no qubits");
    if (nc < 0 || nc > QK_MAX_CONTROLS || !valid_qubits(c, targets, nt) || !valid_qubits(c, controls, nc))
        return fail(c, QK_EINVAL, "apply_gate: bad target or control list");
    for (int a = 0; a < nt; ++a)
        for (int b = 0; b < nc; ++b)
            if (targets[a] == controls[b]) return fail(c, QK_EINVAL, "apply_gate: qubit %d is target and control", targets[a]);
    qk::Cond cond{};
    if (!fill_cond(c, cond, cond_cbits, ncc)) return fail(c, QK_EINVAL, "apply_gate: bad classical condition");
    if (np < 0 || (np > 0 && !params)) return fail(c, QK_EINVAL, "apply_gate: bad params");

    uint64_t cmask = 0;
    for (int b = 0; b < nc; ++b) cmask |= 1ull << c->l2p[controls[b]];

    if (gate_id < 0) {
        cd m[4];
        int ntg = 0;
        if (!qk::builtin_matrix(gate_id, params, np, m, ntg)) return fail(c, QK_EINVAL, "apply_gate: unknown built-in %d or bad params", gate_id);
        if (nt != ntg) return fail(c, QK_EINVAL, "apply_gate: built-in %d takes %d targets", gate_id, ntg);
        if (gate_id == QK_GATE_SWAP) {
            if (nc == 0 && ncc == 0) {
                // SWAP without controls: relabel logical -> physical, no data movement
                qk_status s = QK_OK;
                std::swap(c->l2p[targets[0]], c->l2p[targets[1]]);
                return s;
            }
            // controlled or classically conditioned SWAP: dense 4x4 block
            qk_status s = flush(c);
            if (s != QK_OK) return s;
            qk::MatKArgs a{};
            a.k = 2;
            a.tpos[0] = c->l2p[targets[0]];
            a.tpos[1] = c->l2p[targets[1]];
            a.cmask = cmask;
            std::vector<int> pos{a.tpos[0], a.tpos[1]};
            for (int b = 0; b < nc; ++b) pos.push_back(c->l2p[controls[b]]);
            set_positions(a.ins, pos);
            a.n_groups = 1ull << (c->n - (int)pos.size());
            a.mat = c->d_swap_mat;
            a.cond = cond;
            LaunchScope ls(c, 3, (double)2 * c->amp * (double)(a.n_groups << 2));
            CUDA_TRY(c, qk::launch_matk((int)c->prec, c->d_state, a, c->d_cbits, c->sms, c->stream));
            return QK_OK;
        }
        return apply_1q(c, m, c->l2p[targets[0]], cmask, cond);
    }

    if (gate_id >= (int)c->gates.size()) return fail(c, QK_EINVAL, "apply_gate: unknown gate id %d", gate_id);
    const GateDef &g = c->gates[gate_id];
    if (nt != g.k) return fail(c, QK_EINVAL, "apply_gate: gate %d takes %d targets, got %d", gate_id, g.k, nt);
    if (g.kind == 0) {
        if (g.k == 1) {
            cd m[4] = {g.m[0], g.m[1], g.m[2], g.m[3]};
            return apply_1q(c, m, c->l2p[targets[0]], cmask, cond);
        }
        const int d = 1 << g.k;
        if (g.diagonal) {
            int nonunit = 0;
            for (int x = 0; x < d; ++x) nonunit += (g.m[x * d + x] != 1.0);
            if (nonunit <= 2) {
                for (int x = 0; x < d; ++x) {
                    if (g.m[x * d + x] == 1.0) continue;
                    qk::FusedOp op;
                    op.kind = qk::FusedOp::PHASE;
                    op.mask = cmask;
                    op.val = cmask;
                    for (int a = 0; a < g.k; ++a) {
                        const uint64_t tb = 1ull << c->l2p[targets[a]];
                        op.mask |= tb;
                        if ((x >> (g.k - 1 - a)) & 1) op.val |= tb;
                    }
                    op.f = g.m[x * d + x];
                    op.cond = cond;
                    qk_status s = enqueue(c, op);
                    if (s != QK_OK) return s;
                }
                return QK_OK;
            }
        }
        qk_status s = flush(c);
        if (s != QK_OK) return s;
        if (g.k >= 3 && g.k <= 5 && c->n >= 5 && c->prec == QK_C64 && nc == 0 && ncc == 0 &&
            !c->opt.no_tensor_cores) {
            // targets elsewhere are first gathered onto the lowest physical qubits
            // (one relabelling pass), which costs far less than a CUDA-core block
            // pass; 3- and 4-qubit gates run as 5-qubit blocks U (x) I
            qk_status sm = move_to_low(c, targets, g.k);
            if (sm != QK_OK) return sm;
            uint32_t key = 0;
            for (int a = 0; a < g.k; ++a) key |= (uint32_t)c->l2p[targets[a]] << (3 * a);
            return apply_block_tc(c, gate_id, targets, key);
        }
        qk::MatKArgs a{};
        a.k = g.k;
        std::vector<int> pos;
        for (int t = 0; t < g.k; ++t) {
            a.tpos[t] = c->l2p[targets[t]];
            pos.push_back(a.tpos[t]);
        }
        for (int b = 0; b < nc; ++b) pos.push_back(c->l2p[controls[b]]);
        set_positions(a.ins, pos);
        a.cmask = cmask;
        a.n_groups = 1ull << (c->n - (int)pos.size());
        a.mat = g.d_mat;
        a.cond = cond;
        LaunchScope ls(c, 3, (double)2 * c->amp * (double)(a.n_groups << g.k));
        CUDA_TRY(c, qk::launch_matk((int)c->prec, c->d_state, a, c->d_cbits, c->sms, c->stream));
        return QK_OK;
    }
    // permutation gates: out-of-place gather into scratch, then swap buffers
    qk_status s = flush(c);
    if (s != QK_OK) return s;
    s = ensure_scratch(c);
    if (s != QK_OK) return s;
    qk::PermArgs a{};
    a.w = g.k;
    for (int t = 0; t < g.k; ++t) a.rpos[t] = c->l2p[targets[t]];
    a.field = qk::reg_field_of(a.rpos, g.k);
    a.cmask = cmask;
    a.n_amps = 1ull << c->n;
    a.kind = g.kind == 1 ? 0 : 1;
    a.N = g.N;
    a.cinv = g.cinv;
    a.mu = g.kind == 1 ? (~0ull) / g.N : 0;
    a.finv = g.d_finv;
    a.cond = cond;
    {
        LaunchScope ls(c, 4, (double)2 * c->amp * (double)(1ull << (c->n - nc)));
        CUDA_TRY(c, qk::launch_perm((int)c->prec, c->d_state, c->d_scratch, a, c->d_cbits, c->sms, c->stream));
    }
    std::swap(c->d_state, c->d_scratch);
    return QK_OK;
}

qk_status qk_apply_modexp(qk_ctx *c, const int *targets, int nt, const int *controls, const uint64_t *mult, int nc,
                          uint64_t N, const int *cond_cbits, int ncc) {
    if (!c) return QK_EINVAL;
    if (c->n == 0) return fail(c, QK_ESTATE, "apply_modexp: no qubits");
    if (nt < 1 || nt > QK_MAX_PERM_QUBITS || !valid_qubits(c, targets, nt))
        return fail(c, QK_EINVAL, "apply_modexp: bad target register");
    if (nc < 0 || nc > QK_MAX_MODEXP_CONTROLS || !valid_qubits(c, controls, nc) || (nc > 0 && !mult))
        return fail(c, QK_EINVAL, "apply_modexp: bad control list");
    for (int a = 0; a < nt; ++a)
        for (int b = 0; b < nc; ++b)
            if (targets[a] == controls[b]) return fail(c, QK_EINVAL, "apply_modexp: qubit %d is target and control", targets[a]);
    if (N < 2 || N > (1ull << nt)) return fail(c, QK_EINVAL, "apply_modexp: N=%llu does not fit %d qubits", (unsigned long long)N, nt);
    qk::Cond cond{};
    if (!fill_cond(c, cond, cond_cbits, ncc)) return fail(c, QK_EINVAL, "apply_modexp: bad classical condition");
    std::vector<uint64_t> inv(nc);
    for (int j = 0; j < nc; ++j) {
        if (mult[j] >= N) return fail(c, QK_EINVAL, "apply_modexp: multiplier %d must be < N", j);
        bool ok = false;
        inv[j] = qk::modinv(mult[j], N, ok);
        if (!ok)
            return fail(c, QK_ENOTBIJECTIVE, "x -> %llu x mod %llu is not a permutation (gcd != 1)",
                        (unsigned long long)mult[j], (unsigned long long)N);
    }
    if (nc == 0) return QK_OK;
    qk_status s = flush(c);
    if (s != QK_OK) return s;
    s = ensure_scratch(c);
    if (s != QK_OK) return s;
    thread_local qk::ModExpArgs a;   // 6 KB of tables: built here, copied into the launch
    std::memset(&a, 0, sizeof a);
    a.w = nt;
    for (int t = 0; t < nt; ++t) a.rpos[t] = c->l2p[targets[t]];
    a.field = qk::reg_field_of(a.rpos, nt);
    a.nctl = nc;
    a.ngroups = (nc + 7) / 8;
    for (int j = 0; j < nc; ++j) a.cpos[j] = c->l2p[controls[j]];
    a.n_amps = 1ull << c->n;
    a.N = N;
    a.mu = (~0ull) / N;
    a.cond = cond;
    // group tables: the product of the selected inverses, exact in 64 bits (N <= 2^30)
    for (int g = 0; g < a.ngroups; ++g) {
        const int j0 = 8 * g, nb = std::min(8, nc - j0);
        for (int v = 0; v < (1 << nb); ++v) {
            uint64_t m = 1 % N;
            for (int b = 0; b < nb; ++b)
                if ((v >> b) & 1) m = m * inv[j0 + b] % N;
            a.tab[g][v] = (uint32_t)m;
        }
    }
    {
        LaunchScope ls(c, 4, (double)2 * c->amp * (double)(1ull << c->n));
        CUDA_TRY(c, qk::launch_modexp((int)c->prec, c->d_state, c->d_scratch, a, c->d_cbits, c->sms, c->stream));
    }
    std::swap(c->d_state, c->d_scratch);
    return QK_OK;
}

qk_status qk_apply_gates(qk_ctx *c, const qk_gate_op *ops, int count) {
    if (!c) return QK_EINVAL;
    if (count < 0 || (count > 0 && !ops)) return fail(c, QK_EINVAL, "apply_gates: bad gate list");
    for (int i = 0; i < count; ++i) {
        const qk_gate_op &g = ops[i];
        if (g.nc < 0 || g.nc > 4 || g.ncc < 0 || g.ncc > 4 || g.np < 0 || g.np > 3)
            return fail(c, QK_EINVAL, "apply_gates: entry %d has bad counts", i);
        const qk_status st = qk_apply_gate(c, g.gate_id, &g.target, 1, g.controls, g.nc, g.cond, g.ncc, g.params, g.np);
        if (st != QK_OK) {
            const std::string msg = c->err;
            return fail(c, st, "apply_gates: entry %d: %s", i, msg.c_str());
        }
    }
    return QK_OK;
}

qk_status qk_apply_rphase_cbits(qk_ctx *c, int target, const int *cbits, int ncb) {
    if (!c) return QK_EINVAL;
    if (c->n == 0) return fail(c, QK_ESTATE, "apply_rphase_cbits: no qubits");
    if (target < 0 || target >= c->n) return fail(c, QK_EINVAL, "apply_rphase_cbits: bad target");
    if (ncb < 0 || ncb > QK_MAX_RPHASE_CBITS || (ncb > 0 && !cbits))
        return fail(c, QK_EINVAL, "apply_rphase_cbits: bad cbit list");
    for (int a = 0; a < ncb; ++a)
        if (cbits[a] < 0 || cbits[a] >= c->ncb) return fail(c, QK_EINVAL, "apply_rphase_cbits: cbit %d out of range", cbits[a]);
    if (ncb == 0) return QK_OK;
    qk_status s = flush(c);
    if (s != QK_OK) return s;
    qk::PhaseArgs a{};
    const int q = c->l2p[target];
    a.mask = 1ull << q;
    a.val = 1ull << q;
    set_positions(a.ins, {q});
    a.n_units = 1ull << (c->n - 1);
    a.n_rphase = ncb;
    for (int l = 0; l < ncb; ++l) a.rphase_idx[l] = cbits[l];
    a.f_re = 1.0;
    a.f_im = 0.0;
    LaunchScope ls(c, 2, (double)2 * c->amp * (double)a.n_units);
    CUDA_TRY(c, qk::launch_phase((int)c->prec, c->d_state, a, c->d_cbits, c->sms, c->stream));
    return QK_OK;
}

qk_status qk_apply_kitaev_stage(qk_ctx *c, int control, int gate_id, const int *targets, int nt,
                                const int *phase_cbits, int ncb, double uniform, int dest) {
    if (!c) return QK_EINVAL;
    if (c->n < 2) return fail(c, QK_ESTATE, "kitaev_stage: need at least 2 qubits");
    if (control < 0 || control >= c->n) return fail(c, QK_EINVAL, "kitaev_stage: bad control qubit");
    if (gate_id < 0 || gate_id >= (int)c->gates.size() || c->gates[gate_id].kind == 0)
        return fail(c, QK_EINVAL, "kitaev_stage: gate %d is not a permutation gate", gate_id);
    const GateDef &g = c->gates[gate_id];
    if (nt != g.k || !valid_qubits(c, targets, nt)) return fail(c, QK_EINVAL, "kitaev_stage: bad target list");
    for (int a = 0; a < nt; ++a)
        if (targets[a] == control) return fail(c, QK_EINVAL, "kitaev_stage: control is a target");
    if (ncb < 0 || ncb > QK_MAX_RPHASE_CBITS || (ncb > 0 && !phase_cbits))
        return fail(c, QK_EINVAL, "kitaev_stage: bad phase cbit list");
    for (int a = 0; a < ncb; ++a)
        if (phase_cbits[a] < 0 || phase_cbits[a] >= c->ncb) return fail(c, QK_EINVAL, "kitaev_stage: cbit out of range");
    if (!(uniform >= 0.0 && uniform < 1.0)) return fail(c, QK_EINVAL, "kitaev_stage: uniform not in [0, 1)");
    if (dest < 0 || dest >= c->ncb) return fail(c, QK_EINVAL, "kitaev_stage: destination cbit out of range");
    qk_status s = flush(c);
    if (s != QK_OK) return s;
    s = ensure_scratch(c);
    if (s != QK_OK) return s;
    s = ensure_slots(c, 1);
    if (s != QK_OK) return s;
    qk::KitaevArgs a{};
    a.cpos = c->l2p[control];
    a.w = g.k;
    for (int t = 0; t < g.k; ++t) a.rpos[t] = c->l2p[targets[t]];
    a.field = qk::reg_field_of(a.rpos, g.k);
    a.kind = g.kind == 1 ? 0 : 1;
    a.N = g.N;
    a.cinv = g.cinv;
    a.mu = g.kind == 1 ? (~0ull) / g.N : 0;
    a.finv = g.d_finv;
    a.n_rphase = ncb;
    for (int l = 0; l < ncb; ++l) a.rphase_idx[l] = phase_cbits[l];
    a.n_half = 1ull << (c->n - 1);
    const double half = (double)c->amp * (double)a.n_half;
    {
        LaunchScope ls(c, 4, 2 * half);
        const qk::Decide d{c->d_counter, uniform, c->d_slots, c->d_cbits, dest};
        // half the measurement grid: the stage's state sits in L2 and a longer grid
        // only adds partials for the deciding block to add
        CUDA_TRY(c, qk::launch_kitaev_reduce((int)c->prec, c->d_state, a, c->d_cbits, c->d_partials,
                                             c->meas_blocks / 2, d, c->stream));
    }
    {
        LaunchScope ls(c, 4, 4 * half);
        CUDA_TRY(c, qk::launch_kitaev_update((int)c->prec, c->d_state, c->d_scratch, a, c->d_cbits, c->d_slots, c->sms,
                                             c->stream));
    }
    std::swap(c->d_state, c->d_scratch);
    return QK_OK;
}

qk_status qk_measure(qk_ctx *c, const int *qubits, int nq, const double *uniforms, const int *dest, uint64_t *outcome) {
    if (!c) return QK_EINVAL;
    if (c->n == 0) return fail(c, QK_ESTATE, "measure: no qubits");
    if (nq < 1 || nq > 64 || !valid_qubits(c, qubits, nq) || !uniforms)
        return fail(c, QK_EINVAL, "measure: bad qubit list (1..64 distinct qubits)");
    for (int a = 0; a < nq; ++a) {
        if (!(uniforms[a] >= 0.0 && uniforms[a] < 1.0)) return fail(c, QK_EINVAL, "measure: uniform %d not in [0, 1)", a);
        if (dest && (dest[a] < 0 || dest[a] >= c->ncb)) return fail(c, QK_EINVAL, "measure: destination cbit %d out of range", dest[a]);
    }
    if (outcome && c->capturing) return fail(c, QK_ESTATE, "measure with a host outcome is not allowed while capturing");
    qk_status s = flush(c);
    if (s != QK_OK) return s;
    s = ensure_slots(c, nq);
    if (s != QK_OK) return s;
    // decision k sums over the amplitudes that match decisions 0..k-1 (no
    // collapse in between); one collapse pass projects onto all outcomes at the end
    qk::MeasArgs ma{};
    for (int a = 0; a < nq; ++a) ma.pos[a] = c->l2p[qubits[a]];
    for (int k = 0; k < nq; ++k) {
        ma.k = k;
        ma.nins = k;
        std::vector<int> ins(ma.pos, ma.pos + k);
        std::sort(ins.begin(), ins.end());
        for (int t = 0; t < k; ++t) ma.ins[t] = ins[t];
        ma.n_units = 1ull << (c->n - k);
        {
            LaunchScope ls(c, 5, (double)c->amp * (double)ma.n_units);
            const qk::Decide d{c->d_counter, uniforms[k], c->d_slots + k, c->d_cbits, dest ? dest[k] : -1};
            CUDA_TRY(c, qk::launch_measure_reduce((int)c->prec, c->d_state, c->n, ma, c->d_slots, c->d_partials,
                                                  c->meas_blocks, d, c->stream));
        }
    }
    ma.k = nq;
    {
        LaunchScope ls(c, 5, (double)c->amp * (double)((1ull << c->n) + (1ull << (c->n - nq))));
        CUDA_TRY(c, qk::launch_measure_collapse((int)c->prec, c->d_state, c->n, ma, c->d_slots, c->sms, c->stream));
    }
    if (outcome && c->capturing) return fail(c, QK_ESTATE, "measure with a host outcome is not allowed while capturing");
    if (outcome) {
        std::vector<qk::MeasSlot> h(nq);
        CUDA_TRY(c, cudaMemcpyAsync(h.data(), c->d_slots, sizeof(qk::MeasSlot) * nq, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        uint64_t v = 0;
        for (int a = 0; a < nq; ++a) v = (v << 1) | (uint64_t)(h[a].m & 1);
        *outcome = v;
    }
    return QK_OK;
}

qk_status qk_read_cbits(qk_ctx *c, uint8_t *out, int n) {
    if (!c) return QK_EINVAL;
    NOT_WHILE_CAPTURING(c, "read_cbits");
    if (n < 0 || n > c->ncb || (n > 0 && !out)) return fail(c, QK_EINVAL, "read_cbits: bad count");
    qk_status s = flush(c);
    if (s != QK_OK) return s;
    if (n > 0) CUDA_TRY(c, cudaMemcpyAsync(out, c->d_cbits, n, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return QK_OK;
}

qk_status qk_write_cbits(qk_ctx *c, int first, const uint8_t *in, int n) {
    if (!c) return QK_EINVAL;
    NOT_WHILE_CAPTURING(c, "write_cbits");
    if (first < 0 || n < 0 || first + n > c->ncb || (n > 0 && !in)) return fail(c, QK_EINVAL, "write_cbits: bad range");
    for (int a = 0; a < n; ++a)
        if (in[a] > 1) return fail(c, QK_EINVAL, "write_cbits: values must be 0 or 1");
    qk_status s = flush(c);
    if (s != QK_OK) return s;
    if (n > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(c->d_cbits + first, in, n, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // the host buffer may be pageable
    }
    return QK_OK;
}

qk_status qk_get_state(qk_ctx *c, void *host_out, size_t bytes) {
    if (!c) return QK_EINVAL;
    NOT_WHILE_CAPTURING(c, "get_state");
    if (c->n == 0 || !host_out || bytes != c->state_bytes)
        return fail(c, QK_EINVAL, "get_state: need a buffer of exactly %zu bytes", c->state_bytes);
    qk_status s = flush(c);
    if (s == QK_OK) s = canonicalize(c);
    if (s != QK_OK) return s;
    CUDA_TRY(c, cudaMemcpyAsync(host_out, c->d_state, bytes, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return QK_OK;
}

qk_status qk_set_state(qk_ctx *c, const void *host_in, size_t bytes) {
    if (!c) return QK_EINVAL;
    NOT_WHILE_CAPTURING(c, "set_state");
    if (c->n == 0 || !host_in || bytes != c->state_bytes)
        return fail(c, QK_EINVAL, "set_state: need a buffer of exactly %zu bytes", c->state_bytes);
    c->pending.clear();
    for (int q = 0; q < c->n; ++q) c->l2p[q] = q;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_state, host_in, bytes, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return QK_OK;
}

qk_status qk_reset(qk_ctx *c) {
    if (!c) return QK_EINVAL;
    if (c->n == 0) return fail(c, QK_ESTATE, "reset: no qubits");
    c->pending.clear();
    for (int q = 0; q < c->n; ++q) c->l2p[q] = q;
    CUDA_TRY(c, cudaMemsetAsync(c->d_state, 0, c->state_bytes, c->stream));
    CUDA_TRY(c, qk::launch_set_basis((int)c->prec, c->d_state, 0, c->stream));
    return QK_OK;
}

qk_status qk_device_state(qk_ctx *c, void **dptr, size_t *bytes) {
    if (!c) return QK_EINVAL;
    NOT_WHILE_CAPTURING(c, "device_state");
    if (!dptr || !bytes) return fail(c, QK_EINVAL, "device_state: null output");
    qk_status s = flush(c);
    if (s == QK_OK) s = canonicalize(c);
    if (s != QK_OK) return s;
    *dptr = c->d_state;
    *bytes = c->state_bytes;
    return QK_OK;
}

qk_status qk_flush(qk_ctx *c) {
    if (!c) return QK_EINVAL;
    return flush(c);
}

qk_status qk_sync(qk_ctx *c) {
    if (!c) return QK_EINVAL;
    NOT_WHILE_CAPTURING(c, "sync");
    qk_status s = flush(c);
    if (s != QK_OK) return s;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    int err = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (err) {
        CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
        return fail(c, QK_ETIMEOUT, "a tensor-core pass gave up a bounded wait; the state is not valid");
    }
    return QK_OK;
}

qk_status qk_selftest_timeout(qk_ctx *c) {
    if (!c) return QK_EINVAL;
    NOT_WHILE_CAPTURING(c, "selftest_timeout");
    CUDA_TRY(c, qk::launch_wait_selftest(c->d_err, c->stream));
    return QK_OK;
}

qk_status qk_capture_begin(qk_ctx *c) {
    if (!c) return QK_EINVAL;
    NOT_WHILE_CAPTURING(c, "capture_begin");
    if (c->n == 0) return fail(c, QK_ESTATE, "capture_begin: no qubits");
    qk_status s = flush(c);
    if (s == QK_OK) s = canonicalize(c);
    if (s != QK_OK) return s;
    CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    c->cap_state0 = c->d_state;
    return QK_OK;
}

qk_status qk_capture_end(qk_ctx *c, qk_graph **out) {
    if (!c) return QK_EINVAL;
    if (!c->capturing) return fail(c, QK_ESTATE, "capture_end without capture_begin");
    if (!out) return fail(c, QK_EINVAL, "capture_end: null output");
    *out = nullptr;
    qk_status s = flush(c);
    if (s == QK_OK) s = canonicalize(c);        // back to the identity qubit map
    if (s == QK_OK && c->d_state != c->cap_state0) {
        // an odd number of out-of-place passes: copy back so that replays compose
        if (cudaMemcpyAsync(c->cap_state0, c->d_state, c->state_bytes, cudaMemcpyDeviceToDevice, c->stream) !=
            cudaSuccess)
            s = fail(c, QK_ECUDA, "capture_end: copy-back failed");
        std::swap(c->d_state, c->d_scratch);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    c->capturing = false;
    if (s != QK_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return fail(c, QK_ECUDA, "cudaStreamEndCapture failed: %s", cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e2 = cudaGraphInstantiate(&exec, graph, 0);
    if (e2 != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(c, QK_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e2));
    }
    qk_graph *g = new (std::nothrow) qk_graph{c, graph, exec};
    if (!g) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return fail(c, QK_ENOMEM, "capture_end: out of host memory");
    }
    *out = g;
    return QK_OK;
}

qk_status qk_graph_launch(qk_graph *g) {
    if (!g) return QK_EINVAL;
    qk_ctx *c = g->ctx;
    NOT_WHILE_CAPTURING(c, "graph_launch");
    qk_status s = flush(c);
    if (s == QK_OK) s = canonicalize(c);   // the graph expects the identity map
    if (s != QK_OK) return s;
    CUDA_TRY(c, cudaGraphLaunch(g->exec, c->stream));
    return QK_OK;
}

qk_status qk_graph_destroy(qk_graph *g) {
    if (!g) return QK_EINVAL;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return QK_OK;
}

int qk_num_qubits(const qk_ctx *c) { return c ? c->n : -1; }
int qk_num_cbits(const qk_ctx *c) { return c ? c->ncb : -1; }

qk_status qk_get_counters(const qk_ctx *c, uint64_t *launches, uint64_t *passes, uint64_t *bytes) {
    if (!c) return QK_EINVAL;
    if (launches) *launches = c->launches;
    if (passes) *passes = c->passes_x1000 / 1000;
    if (bytes) *bytes = (uint64_t)c->alg_bytes;
    return QK_OK;
}

qk_status qk_reset_counters(qk_ctx *c) {
    if (!c) return QK_EINVAL;
    c->launches = 0;
    c->passes_x1000 = 0;
    c->alg_bytes = 0;
    return QK_OK;
}

qk_status qk_profile(qk_ctx *c, uint64_t launches[QK_NUM_LAUNCH_CLASSES], double ms[QK_NUM_LAUNCH_CLASSES],
                     double bytes[QK_NUM_LAUNCH_CLASSES]) {
    if (!c) return QK_EINVAL;
    if (!c->opt.profile) return fail(c, QK_ESTATE, "profile: context created without options.profile");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (auto &p : c->prof) {
        float t = 0.f;
        CUDA_TRY(c, cudaEventElapsedTime(&t, p.a, p.b));
        c->prof_launches[p.cls]++;
        c->prof_ms[p.cls] += t;
        c->prof_bytes[p.cls] += p.bytes;
        c->ev_pool.push_back(p.a);
        c->ev_pool.push_back(p.b);
    }
    c->prof.clear();
    for (int k = 0; k < QK_NUM_LAUNCH_CLASSES; ++k) {
        if (launches) launches[k] = c->prof_launches[k];
        if (ms) ms[k] = c->prof_ms[k];
        if (bytes) bytes[k] = c->prof_bytes[k];
        c->prof_launches[k] = 0;
        c->prof_ms[k] = 0;
        c->prof_bytes[k] = 0;
    }
    return QK_OK;
}

const char *qk_last_error(const qk_ctx *c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
