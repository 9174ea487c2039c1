// Internal declarations shared by the libqk host code and its CUDA kernels.
// Nothing here is part of the public ABI (include/qk.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace qk {

constexpr int kMaxPos = 24;        // sorted bit positions a launch may insert
constexpr int kMaxCond = 16;       // classical-condition cbits per gate
constexpr int kMaxRphase = 62;     // cbits feeding one semiclassical phase
constexpr int kMaxPermW = 30;      // permutation register width

// Classical condition: the launch acts only if every listed cbit is 1.
struct Cond {
    int n;
    int idx[kMaxCond];
};

// Sorted ascending bit positions, used to enumerate a subspace by inserting a
// bit at each position into a dense counter.
struct Positions {
    int n;
    int pos[kMaxPos];
};

// 2x2 update on target bit q where all control bits (cmask) are 1.
struct U2Args {
    double m[8];          // m00, m01, m10, m11 as (re, im) pairs, FP64 master
    uint64_t cmask;
    int q;
    Positions ins;        // q and every control, sorted
    uint64_t n_units;     // work units in the subspace
    Cond cond;
};

// Multiply amplitudes whose index satisfies (i & mask) == val by f.
struct PhaseArgs {
    double f_re, f_im;
    uint64_t mask, val;
    Positions ins;        // bits of mask, sorted
    uint64_t n_units;
    Cond cond;
    // semiclassical phase (rphase): when n_rphase > 0, f is computed on the
    // device as exp(-2 pi i sum_l c[rphase_idx[l-1]] / 2^(l+1)).
    int n_rphase;
    int rphase_idx[kMaxRphase];
};

// Dense k-qubit matrix on arbitrary targets with controls.
struct MatKArgs {
    int k;
    int tpos[8];          // physical bit of register bit (k-1-a), a = list index; tpos[0] = MSB
    uint64_t cmask;
    Positions ins;        // targets and controls, sorted
    uint64_t n_groups;
    const void *mat;      // device matrix, 2^k x 2^k, row-major, amplitude type
    Cond cond;
};

// Controlled permutation of a w-bit register, out-of-place gather.
// A register whose qubits sit on consecutive physical bits p0 .. p0 + w - 1 is a bit
// field of the index: its value is the field itself (first-listed qubit highest,
// rev = 0) or the field bit-reversed (first-listed qubit lowest, rev = 1).  Kernels
// use the field form when contig is set and the per-bit gather otherwise.
struct RegField {
    int contig, p0, rev;
};
inline RegField reg_field_of(const int *rpos, int w) {
    RegField f{0, 0, 0};
    bool asc = true, desc = true;
    for (int t = 0; t < w; ++t) {
        asc = asc && rpos[t] == rpos[0] + t;
        desc = desc && rpos[t] == rpos[0] - t;
    }
    if (w >= 1 && asc) f = RegField{1, rpos[0], 1};
    else if (w >= 1 && desc) f = RegField{1, rpos[w - 1], 0};
    return f;
}
#ifdef __CUDACC__
__device__ __forceinline__ uint64_t field_get(uint64_t i, const RegField &f, int w) {
    const uint64_t v = (i >> f.p0) & ((1ull << w) - 1);
    return f.rev ? (__brevll(v) >> (64 - w)) : v;
}
__device__ __forceinline__ uint64_t field_put(uint64_t i, uint64_t x, const RegField &f, int w) {
    const uint64_t v = f.rev ? (__brevll(x) >> (64 - w)) : x;
    const uint64_t m = ((1ull << w) - 1) << f.p0;
    return (i & ~m) | (v << f.p0);
}
#endif

struct PermArgs {
    int w;
    int rpos[kMaxPermW];  // physical bit of register list entry a (a = 0 is the MSB)
    RegField field;       // zero (per-bit gather) unless set from rpos
    uint64_t cmask;
    uint64_t n_amps;
    int kind;             // 0 = mul-mod, 1 = table
    uint64_t N, cinv, mu; // mul-mod: y -> cinv*y mod N for y < N, mu = floor((2^64-1)/N)
    const uint32_t *finv; // table: inverse permutation
    Cond cond;
};

// Modular exponentiation of a register by a control register: for each basis
// state, the register value x < N becomes M x mod N, M the product of the
// multipliers whose control qubits are 1 (x >= N is left alone).  The controls go
// in groups of 8; tab[g][v] is the inverse of the product of group g's
// multipliers selected by the bits of v (the gather reads x = M^-1 y).
constexpr int kModExpMaxControls = 48;
constexpr int kModExpGroups = kModExpMaxControls / 8;
struct ModExpArgs {
    int w;
    int rpos[kMaxPermW];  // physical bit of register list entry a (a = 0 is the MSB)
    RegField field;       // zero (per-bit gather) unless set from rpos
    int nctl, ngroups;
    int cpos[kModExpMaxControls];   // physical bit of control j (group j / 8, bit j % 8)
    uint64_t n_amps;
    uint64_t N, mu;       // mu = floor((2^64-1)/N)
    Cond cond;
    uint32_t tab[kModExpGroups][256];
};

// Device-side record of one single-qubit measurement decision.
struct MeasSlot {
    double p0;            // probability of reading 0
    double scale;         // 1/sqrt(P_m)
    int m;                // outcome
    int pad;
};

// Where a reduction's decision goes.  Every block of the reduction stores its
// (S0, S1) partials; the last block to finish (an atomic ticket, no waiting) adds
// all partials in a fixed order, so the result does not depend on timing, and
// records P0 = S0 / (S0 + S1), the outcome m = (u >= P0), 1/sqrt(S_m) and the cbit.
struct Decide {
    unsigned *counter;    // zero between launches; the deciding block resets it
    double u;
    MeasSlot *slot;
    uint8_t *cbits;
    int dest;             // destination cbit, -1: none
};
#ifdef __CUDACC__
// Running sum of FP32 terms kept as an unevaluated pair hi + lo (Knuth's TwoSum:
// the rounding error of each addition is carried in lo): about twice float's
// precision at the FP32 rate.  GB300's FP64 rate is too low for an FP64 add per
// term (2 FP64 lanes per SM per clock).
struct FSum {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float s = hi + x;
        const float bp = s - hi;
        const float e = (hi - (s - bp)) + (x - bp);
        hi = s;
        lo += e;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Sum over the block of one double per thread, the FP64 additions done by warp 0
// alone; sh holds blockDim.x doubles.  The result is valid in thread 0.
__device__ __forceinline__ double block_sum_w0(double v, double *sh) {
    __syncthreads();
    sh[threadIdx.x] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        for (int k = threadIdx.x; k < (int)blockDim.x; k += 32) t += sh[k];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

// Called by every thread of every block after thread 0 stored the block's
// partials[2 * blockIdx.x + {0, 1}].
__device__ __forceinline__ void last_block_decides(double *partials, const Decide &d) {
    __shared__ unsigned s_last;
    __shared__ double s_sum[2][32];
    if (threadIdx.x == 0) {
        __threadfence();                     // the partials before the ticket
        s_last = atomicAdd(d.counter, 1u) == gridDim.x - 1 ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double a0 = 0.0, a1 = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        a0 += __ldcg(&partials[2 * b]);
        a1 += __ldcg(&partials[2 * b + 1]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_sum[0][threadIdx.x >> 5] = a0;
        s_sum[1][threadIdx.x >> 5] = a1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s0 += s_sum[0][w];
            s1 += s_sum[1][w];
        }
        const double tot = s0 + s1;
        const double p0 = tot > 0.0 ? s0 / tot : 1.0;
        const int m = (d.u >= p0) ? 1 : 0;
        const double pm = m ? s1 : s0;
        d.slot->p0 = p0;
        d.slot->m = m;
        d.slot->scale = pm > 0.0 ? 1.0 / sqrt(pm) : 0.0;
        if (d.dest >= 0) d.cbits[d.dest] = (uint8_t)m;
        *d.counter = 0;
    }
}
#endif

// Measurement of a list of qubits, one decision at a time.  Decision k sums
// |a_i|^2 over the indices whose earlier measured bits equal the outcomes
// already decided (read from the slots on the device), split by bit pos[k].
constexpr int kMaxMeasure = 64;
struct MeasArgs {
    int k;                // decisions already taken (prefix length); collapse: all decisions
    int pos[40];          // physical bit of measured qubit j (list order), j < k and j == k
    int nins;             // prefix bits sorted ascending, for enumeration
    int ins[40];
    uint64_t n_units;     // 2^(n-k) amplitudes match the prefix
};

// One fused Kitaev stage (kernels_kitaev.cu): control qubit at physical bit
// cpos, register of w qubits at rpos[] (rpos[0] = MSB), permutation f given by
// its inverse (mul-mod: cinv, N, mu; table: finv), phase from cbits.
struct KitaevArgs {
    int cpos;
    int w;
    int rpos[kMaxPermW];
    RegField field;
    int kind;             // 0 = mul-mod, 1 = table
    uint64_t N, cinv, mu;
    const uint32_t *finv;
    int n_rphase;
    int rphase_idx[kMaxRphase];
    uint64_t n_half;      // 2^(n-1): amplitudes with the control bit 0
};

// Qubit-relabelling gather: out[logical index] = in[physical index].
struct RelabelArgs {
    int n;
    int phys_of[40];      // physical bit of logical qubit
    uint64_t n_amps;
};

// ---------------------------------------------------------------------------
// fused tile pass (K3), complex64.  A tile is 2^13 amplitudes over 13 physical
// qubits S[0..12] (S[b] = b for b < 5, so 32 consecutive amplitudes form the
// lane dimension of every global access).  256 threads hold 32 amplitudes each
// in registers; three fixed "arrangements" say which local bits are register,
// lane and warp bits:
//   ARR_IO: lanes = local 0..4, registers = local 5..9,  warps = local 10..12
//   ARR_LO: registers = local 0..4, lanes = local 5..9,  warps = local 10..12
//   ARR_HI: lanes = local 0..4, registers = local 8..12, warps = local 5..7
// Gates act on register bits only; switching arrangement is a transpose through
// shared memory.  Loads use ARR_IO, stores use ARR_IO or ARR_HI.
// ---------------------------------------------------------------------------
constexpr int kTileQubits = 13;
// Physical qubits 0 .. kTileContig-1 belong to every tile pass, so a warp's loads
// and stores touch runs of 2^kTileContig contiguous amplitudes; the other tile
// qubits are chosen freely by the planner.  With 3 the layered 30-qubit circuit
// needs 10 passes instead of 15 but takes as long: the pass is bound by
// instruction issue, and its HBM traffic already overlaps the gate arithmetic.
constexpr int kTileContig = 5;
constexpr int kTileThreads = 256;
constexpr int kTileMaxOps = 192;
constexpr int kTileMaxLin = 512;
// runs of consecutive fixed qubits: S holds 0..4 and eight more bits, which
// split the rest into at most nine runs
constexpr int kTileMaxRuns = 12;
constexpr int kTileMaxMats = 160;
constexpr int kTileMaxConds = 4;
enum TileArr : uint8_t { ARR_IO = 0, ARR_LO = 1, ARR_HI = 2 };
// TOP_U2L: a layer of uncontrolled 2x2 gates on distinct register bits (k is
// the bit mask), in pivot form; their coefficients are lg[first...] in bit order,
// and bit b of rmask says that the gate on register bit b updates the pair's
// stored |0> value first (LayerGate).  After the gates, a CZ between register
// bits (k, l) for every bit set in tmask (bit cz_index(k, l) over the ten pairs,
// see below).
// TOP_PHASEL: a group of thread- or tile-dependent diagonal terms that all add to
// one pending phase sum (register bit k, or the thread constant when k == 5):
// lin[first, first + count), evaluated in place (see LinTerm); rval = 1 says that
// bit k's qubit is stored flipped, so the sum lands on k = 0.  Diagonal terms
// that are the same for every amplitude pair of a qubit (no thread or fixed-bit
// condition) never reach the device: the planner folds them into the next layer
// gate's coefficients or into the final flush.
// TOP_PAIR: factor on the amplitudes whose register bits k and l (code k | l <<
// 3) have the values in rval (bit 0: k, bit 1: l), under the op's thread /
// fixed-bit conditions.
// TOP_PAIRNEG: an unconditional sign flip of the amplitudes whose register bits k
// and l are both 1 (code k | l << 3): a CZ between two register bits.
// TOP_PHASEB: a TOP_PHASEL group whose terms each test one bit (so every term is
// "add turns where the bit is 1"; a term on a bit being 0 was split by the planner
// into a constant it keeps and a negated bit-1 term): count thread-bit terms
// followed by count2 tile-index-bit terms, BitTerm entries from index first of the
// lin[] storage read as BitTerms (two per LinTerm slot); rval as for TOP_PHASEL.
// TOP_PAIRU: a TOP_PAIR without thread, tile or classical condition (the common
// case: a controlled phase between two register bits), always on the stored
// pattern (1, 1): for qubits stored flipped the planner rewrites the factor as a
// (1, 1) factor and uniform single-bit and constant phases.
enum TileOpKind : uint8_t {
    TOP_U2 = 0, TOP_PHASE = 1, TOP_XPOSE = 2, TOP_PHASEB = 3, TOP_U2L = 4, TOP_PAIR = 5, TOP_PHASEL = 6,
    TOP_PAIRNEG = 7, TOP_PAIRU = 8
};
struct BitTerm {
    uint32_t bit;          // thread-bit index (lane 0..4, warp 5..7) or tile-index bit
    uint32_t turns;
};
// the pairs k < l of register bits in the order (0,1) (0,2) (0,3) (0,4) (1,2)
// (1,3) (1,4) (2,3) (2,4) (3,4): the bit of a TOP_U2L op's CZ mask
__host__ __device__ constexpr int cz_index(int k, int l) { return k == 0 ? l - 1 : k == 1 ? l + 2 : k == 2 ? l + 4 : 9; }

// A diagonal term of a TOP_PHASEL group: adds turns where the thread bits match
// (tbits & tmask) == tval and the tile index matches (tile & fmask) == fval (its
// bit b is the fixed qubit fixed[b]).
struct LinTerm {
    uint16_t tmask, tval;
    uint32_t fmask, fval;
    uint32_t turns;
};

// One gate of a TOP_U2L layer in pivot form.  The planner may keep a local
// qubit's two values stored swapped ("flipped"); it picks the stored order of the
// gate's output so that, with M the gate in stored order and the pending factor F
// of the bit folded in, M diag(1, F) has its larger entries on the diagonal
// (|M00| = |M11| >= |M10| = |M01|).  With a0 = M01 F / M00, a1 = M10 / (M11 F)
// the true outputs are (M00 z0, M11 F z1) for z0 = y0 + a0 y1, z1 = y1 + a1 y0.
// The device forms them in place from one value of the pair to the other, 8
// FP32 FMAs per pair:
//   zf = 0:  y1 += a1 y0,  then y0 += s a0 y1   (y0 ends as s z0, y1 as z1)
//   zf = 1:  y0 += a0 y1,  then y1 += s a1 y0   (y0 ends as z0, y1 as s z1)
// with s = 1 / (1 - a0 a1).  For a unitary M, a0 a1 = -|M01|^2 / |M00|^2, so s
// = |M00|^2 is real and in [1/2, 1]; the planner keeps the leftover factor (M00 /
// s and M11 F, or M00 and M11 F / s) as pending: a real scale and a phase for the
// whole pass, and a factor of magnitude in [1/2, 2] on the bit's |1> (it picks zf
// per gate so that the magnitude stays there).  The device uses c0 = C0 e and
// c1 = C1 conj(e), with e the thread-dependent part of F; c[] holds C0 (s a0 or
// a0) and C1 (a1 or s a1) as FFMA2 operand pairs (re, re), (im, im), (-im, -im).
struct LayerGate {
    float2 c[6];           // C0r, C0i, -C0i, C1r, C1i, -C1i, each splatted
};

struct TileOp {
    uint8_t kind;          // TileOpKind
    uint8_t k;             // U2: target register bit; XPOSE: new arrangement
    uint8_t rmask, rval;   // condition on register bits (5-bit register index space)
    uint16_t tmask, tval;  // condition on thread bits: bits 0..4 lane, 5..7 warp
    uint16_t cond;         // index into TileParams::conds, 0xffff = unconditional
    uint16_t count;        // TOP_U2L: gates from lg[first]; TOP_PHASEL: terms from lin[first]
    uint16_t first;
    uint16_t count2;
    uint32_t hturns;       // TOP_U2: uniform pending turns of the target's qubit, added
                           // to the thread's pending sum before the op
    float hmag;            // TOP_U2: uniform pending magnitude of the target's |1>,
                           // applied to the amplitudes before the op (1: none)
    uint64_t gmask, gval;  // condition on the tile's fixed (non-tile) physical bits
    union {
        float m[8];        // U2: m00, m01, m10, m11 as (re, im)
        struct {
            float re, im;  // PHASE: factor f = exp(2 pi i turns / 2^32)
            uint32_t turns;
        } ph;
    };
};
// The tile kernel reads the fields the common op kinds need (kind, k, rval,
// tmask, count, first, count2) as the op's first two 8-byte words, one op ahead.
static_assert(offsetof(TileOp, kind) == 0 && offsetof(TileOp, k) == 1 && offsetof(TileOp, rval) == 3 &&
                  offsetof(TileOp, tmask) == 4 && offsetof(TileOp, count2) == 14 &&
                  offsetof(TileOp, count) == 10 && offsetof(TileOp, first) == 12 && offsetof(TileOp, hturns) == 16,
              "TileOp head layout");
static_assert(alignof(TileOp) >= 8, "TileOp head is read as 8-byte words");

// The scalar part of a tile-pass program (the arrays follow in TileParams, or
// sit in device pools for a batched launch, see TileProg).
struct TileHead {
    uint64_t n_tiles;
    int n;
    int nfix;
    int8_t S[16];          // physical qubit of local bit b
    int8_t fixed[40];      // physical bits of the tile index, ascending
    // the same as runs of consecutive physical bits: tile-index bits [tlo, tlo +
    // len) land on physical bits [plo, plo + len)
    int nruns;
    uint8_t run_tlo[kTileMaxRuns], run_len[kTileMaxRuns], run_plo[kTileMaxRuns];
    int store_arr;
    int n_conds;
    Cond conds[kTileMaxConds];
    int nops;
    // final flush: the uniform pending factor of each local qubit's |1> (phase in
    // turns and magnitude), the uniform constant phase (fin_turns[13]) and the real
    // scale; a plan's last pass also applies the factors that earlier passes left on
    // qubits outside its S: fin_fixed[b] turns and fin_fixed_mag[b] where tile-index
    // bit b (qubit fixed[b]) is 1, for the bits set in fin_fixed_mask
    uint32_t fin_turns[14];
    float fin_mag[kTileQubits];
    float fin_scale;
    int need_tab;          // 0: every phase the pass can form is 0 or half a turn
    uint64_t fin_fixed_mask;
    uint32_t fin_fixed[40];
    float fin_fixed_mag[40];
    int fin_flip;          // local qubits stored flipped at the end (bit b: local qubit b)
    int nlg, nlin;         // entries of lg[] and lin[] in use
};

// A whole pass program, passed as kernel parameters for one state.
struct TileParams : TileHead {
    TileOp ops[kTileMaxOps];
    LayerGate lg[kTileMaxMats];
    LinTerm lin[kTileMaxLin];
};

// A pass program of one circuit in a batched launch: the header plus offsets
// of its ops, layer gates and linear terms in device pools, and its state.
struct TileProg : TileHead {
    uint32_t op0, lg0, lin0, pad;
    float2 *psi;
};
static_assert(sizeof(TileParams) <= 32764, "tile program must fit in the kernel parameter space");

cudaError_t launch_tile(void *psi, const TileParams &p, const uint8_t *cbits, cudaStream_t s);
// Pass k of many circuits in one launch: CTA b runs tile (b - first[c]) of
// program c, where first[] (n_progs + 1 entries, ascending, first[0] = 0) splits
// the grid; programs are in n-qubit order so that the 32-bit offset kernel serves
// every circuit below 33 qubits.
// general: some program holds general ops (see tile_ops_need_general); without
// them a leaner instance of the kernel runs.
cudaError_t launch_tile_batch(const TileProg *progs, const uint32_t *first, int n_progs, uint32_t n_ctas,
                              const TileOp *ops, const LayerGate *lg, const LinTerm *lin, bool general,
                              cudaStream_t s);
// whether a pass program holds ops of the kinds TOP_U2, TOP_PHASE or TOP_PAIR
bool tile_ops_need_general(const TileOp *ops, size_t n);

// ---------------------------------------------------------------------------
// launchers (kernels_basic.cu); prec: 0 = complex64, 1 = complex128
// ---------------------------------------------------------------------------
cudaError_t launch_u2(int prec, void *psi, const U2Args &a, const uint8_t *cbits, int n, int sms,
                      cudaStream_t s);
cudaError_t launch_phase(int prec, void *psi, const PhaseArgs &a, const uint8_t *cbits, int sms,
                         cudaStream_t s);
cudaError_t launch_matk(int prec, void *psi, const MatKArgs &a, const uint8_t *cbits, int sms,
                        cudaStream_t s);
cudaError_t launch_modexp(int prec, const void *in, void *out, const ModExpArgs &a, const uint8_t *cbits, int sms,
                          cudaStream_t s);
cudaError_t launch_perm(int prec, const void *in, void *out, const PermArgs &a, const uint8_t *cbits,
                        int sms, cudaStream_t s);
cudaError_t launch_measure_reduce(int prec, const void *psi, int n, const MeasArgs &a, const MeasSlot *slots,
                                  double *partials, int nblocks, const Decide &d, cudaStream_t s);
cudaError_t launch_measure_collapse(int prec, void *psi, int n, const MeasArgs &a, const MeasSlot *slots, int sms,
                                    cudaStream_t s);
cudaError_t launch_kitaev_reduce(int prec, const void *psi, const KitaevArgs &a, const uint8_t *cbits,
                                 double *partials, int nblocks, const Decide &d, cudaStream_t s);
cudaError_t launch_kitaev_update(int prec, const void *psi, void *out, const KitaevArgs &a, const uint8_t *cbits,
                                 const MeasSlot *slot, int sms, cudaStream_t s);
// K4 on tensor cores (kernels_block_tc.cu): dense 5-qubit complex64 unitary on
// physical qubits 0..4; bh/bl are the 64 x 64 split real embedding (row = output
// column); err receives 1 if a bounded wait gave up.
cudaError_t launch_block_tc(void *psi, int n, const float *bh, const float *bl, int *err, int sms, cudaStream_t s);
// one bounded mbarrier wait that runs out; sets *err (the timeout path's self-test)
cudaError_t launch_wait_selftest(int *err, cudaStream_t s);
cudaError_t launch_set_basis(int prec, void *psi, uint64_t index, cudaStream_t s);
cudaError_t launch_relabel(int prec, const void *in, void *out, const RelabelArgs &a, int sms,
                           cudaStream_t s);

}  // namespace qk
