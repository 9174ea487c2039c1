// Planner for the fused mode: groups queued gates into tile passes (K3).
//
// Two gates commute when neither one's non-diagonal qubit (the target of a 2x2
// gate) is touched by the other; diagonal gates and the control qubits of a
// controlled gate act diagonally.  A pass picks a set S of 13 physical qubits
// (always 0 .. kTileContig-1, for coalesced access) and takes, in order, every
// queued gate that
//   - is diagonal, or is a 2x2 gate whose target is in S (controls may be
//     anywhere: a control outside S is constant over a tile), and
//   - commutes with every earlier gate the pass leaves behind.
// Qubits join S greedily as 2x2 targets are met.  Inside the pass the taken
// gates are list-scheduled over the three register arrangements of the tile
// kernel, inserting a transpose when no ready gate fits the current one.
//
// A last walk over the program (fold_program) turns each layer gate into pivot
// form (LayerGate in qk_kernels.cuh) and keeps, in double precision, every
// pending factor that is the same for all threads -- per local qubit (a phase and
// a magnitude), plus a constant phase -- and the pass's real scale: those fold
// into later gates' coefficients and the final flush, so the device never sees
// them.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <complex>
#include <cstring>
#include <vector>

#include "qk_plan.h"

namespace qk {

struct TilePlanner {
    bool log = false;  // QK_PLAN_LOG=1: one line per tile pass on stderr
};

TilePlanner *make_planner() {
    TilePlanner *p = new TilePlanner();
    const char *e = std::getenv("QK_PLAN_LOG");
    p->log = e && e[0] == '1';
    return p;
}
void free_planner(TilePlanner *p) { delete p; }

namespace {

struct POp {
    const FusedOp *op;
    uint64_t nd;   // non-diagonal qubits
    uint64_t all;  // every qubit the op depends on
};

POp classify(const FusedOp &op) {
    POp p;
    p.op = &op;
    if (op.kind == FusedOp::U2) {
        p.nd = 1ull << op.q;
        p.all = p.nd | op.cmask;
    } else {
        p.nd = 0;
        p.all = op.mask;
    }
    return p;
}

bool commute(const POp &a, const POp &b) { return !(a.nd & b.all) && !(b.nd & a.all); }

bool same_cond(const Cond &a, const Cond &b) {
    if (a.n != b.n) return false;
    for (int k = 0; k < a.n; ++k)
        if (a.idx[k] != b.idx[k]) return false;
    return true;
}

// slot of a local bit in an arrangement: 0 = register, 1 = lane, 2 = warp; *pos = index
int slot_of(int arr, int lb, int *pos) {
    if (arr == ARR_IO) {
        if (lb < 5) { *pos = lb; return 1; }
        if (lb < 10) { *pos = lb - 5; return 0; }
        *pos = lb - 10;
        return 2;
    }
    if (arr == ARR_LO) {
        if (lb < 5) { *pos = lb; return 0; }
        if (lb < 10) { *pos = lb - 5; return 1; }
        *pos = lb - 10;
        return 2;
    }
    // ARR_HI
    if (lb < 5) { *pos = lb; return 1; }
    if (lb < 8) { *pos = lb - 5; return 2; }
    *pos = lb - 8;
    return 0;
}

bool executable(const POp &p, int arr, const int *local_of) {
    if (p.op->kind != FusedOp::U2) return true;
    int pos;
    return slot_of(arr, local_of[p.op->q], &pos) == 0;
}

// Encode a mask/value condition over physical qubits into register / thread /
// fixed-bit parts for an arrangement.
void encode_cond(uint64_t mask, uint64_t val, int arr, const int *local_of, TileOp &t) {
    t.rmask = t.rval = 0;
    t.tmask = t.tval = 0;
    t.gmask = t.gval = 0;
    for (int b = 0; b < 64; ++b) {
        if (!((mask >> b) & 1)) continue;
        const int bit = (int)((val >> b) & 1);
        const int lb = local_of[b];
        if (lb < 0) {
            t.gmask |= 1ull << b;
            t.gval |= (uint64_t)bit << b;
            continue;
        }
        int pos;
        const int s = slot_of(arr, lb, &pos);
        if (s == 0) {
            t.rmask |= (uint8_t)(1 << pos);
            t.rval |= (uint8_t)(bit << pos);
        } else if (s == 1) {
            t.tmask |= (uint16_t)(1 << pos);
            t.tval |= (uint16_t)(bit << pos);
        } else {
            t.tmask |= (uint16_t)(1 << (5 + pos));
            t.tval |= (uint16_t)(bit << (5 + pos));
        }
    }
}

uint32_t angle_turns(double x) {
    double frac = x / (2.0 * M_PI);
    frac -= std::floor(frac);
    return (uint32_t)(uint64_t)std::llround(frac * 4294967296.0);
}
double turns_angle(uint32_t t) { return 2.0 * M_PI * (double)t / 4294967296.0; }

// local qubit of register bit k in an arrangement
int local_of_reg(int arr, int k) { return arr == ARR_IO ? 5 + k : arr == ARR_LO ? k : 8 + k; }

// Planner-only op kind: a diagonal term that is the same for every thread and
// tile (no thread or fixed-bit condition) on register bit k (k == 5: constant),
// ph.turns; fold_program absorbs it and it never reaches the device.
constexpr uint8_t TOP_HOSTPH = 0x40;

using cdm = std::complex<double>;
struct Mat2 {
    cdm m[4];
};

// The program's pending state that is the same for every thread, in double
// precision: mag[q] e^{i u[q]} the factor of local qubit q's stored |1> relative
// to its stored |0>, u0 a constant phase, lam the real scale that the pivot form
// leaves over, flip[q] whether q's values are stored swapped.
struct UniformPending {
    double u[kTileQubits] = {};     // phase of the pending factor on a local qubit's stored |1>
    double mag[kTileQubits];        // its magnitude (in [1/2, 2])
    double u0 = 0.0;
    double lam = 1.0;
    int flip[kTileQubits] = {};   // local qubit stored with its two values swapped
    UniformPending() {
        for (double &m : mag) m = 1.0;
    }
};

// Pivot form of a layer gate on local qubit q (LayerGate in qk_kernels.cuh).  The
// gate in stored order is W = U X^f (f: q stored flipped); the output is stored
// flipped (f') when that puts the larger entries of M = X^f' W on the diagonal.
// F = mag[q] e^{i u[q]} is the pending factor of q's stored |1>.  Returns zf, the
// value of the pair the device updates first: the one that keeps the pending
// magnitude of q's |1> within [1/2, 2] (zf = 0 multiplies it by s <= 1, zf = 1
// divides it by s >= 1/2).
int pivot_gate(const Mat2 &g, UniformPending &st, int q, LayerGate &out) {
    cdm W[4] = {g.m[0], g.m[1], g.m[2], g.m[3]};
    if (st.flip[q]) {  // U X: swap the columns
        std::swap(W[0], W[1]);
        std::swap(W[2], W[3]);
    }
    const bool fout = std::abs(W[0]) < std::abs(W[2]);
    if (fout) {        // X W: swap the rows
        std::swap(W[0], W[2]);
        std::swap(W[1], W[3]);
    }
    const cdm m00 = W[0], m01 = W[1], m10 = W[2], m11 = W[3];
    const cdm F = std::polar(st.mag[q], st.u[q]);
    const cdm A0 = m01 * F / m00, A1 = m10 / (m11 * F);
    // y1 += a1 y0 then y0 += s a0 y1 leaves y0 = s z0 (and the other order y1 =
    // s z1) for s = 1 / (1 - a0 a1), real and in [1/2, 1] for a unitary gate
    const cdm s = 1.0 / (1.0 - A0 * A1);
    const int zf = st.mag[q] < 1.0 ? 1 : 0;
    const cdm C0 = zf ? A0 : s * A0, C1 = zf ? s * A1 : A1;
    const cdm P0 = zf ? m00 : m00 / s, P1 = zf ? m11 * F / s : m11 * F;   // the true outputs' factors
    st.u0 += std::arg(P0);
    st.lam *= std::abs(P0);
    const cdm R = P1 / P0;
    st.u[q] = std::arg(R);
    st.mag[q] = std::abs(R);
    st.flip[q] = fout ? 1 : 0;
    const float a0r = (float)C0.real(), a0i = (float)C0.imag(), a1r = (float)C1.real(), a1i = (float)C1.imag();
    out.c[0] = make_float2(a0r, a0r);
    out.c[1] = make_float2(a0i, a0i);
    out.c[2] = make_float2(-a0i, -a0i);
    out.c[3] = make_float2(a1r, a1r);
    out.c[4] = make_float2(a1i, a1i);
    out.c[5] = make_float2(-a1i, -a1i);
    return zf;
}

// local qubits of the thread bits (0..4 lanes, 5..7 warps) in an arrangement
int local_of_tbit(int arr, int t) {
    if (t < 5) return arr == ARR_LO ? 5 + t : t;
    return arr == ARR_HI ? 5 + (t - 5) : 10 + (t - 5);
}
}  // namespace

qk_status plan_passes(TilePlanner *planner, int n, const std::vector<FusedOp> &ops, const PassSink &sink,
                      const char **err) {
    *err = "";
    std::vector<POp> rem;
    rem.reserve(ops.size());
    for (const auto &op : ops) rem.push_back(classify(op));

    // take limits per pass; halved and retried when a program overflows the
    // kernel-parameter budget (ops and grouped phase entries)
    int max_u2 = 100, max_ph = 300;
    std::vector<POp> left, taken;
    // the uniform pending factors one pass leaves to the next (FP64): per physical
    // qubit, on its |1> (a phase and a magnitude), plus a constant phase and a real
    // scale; only the plan's last pass applies them to the amplitudes
    double carry[64] = {0.0};
    double carry_mag[64];
    for (double &m : carry_mag) m = 1.0;
    double carry_u0 = 0.0, carry_lam = 1.0;
    // The gates one pass takes from rem for a qubit set S: in order, each gate
    // that commutes with every gate left behind before it, whose 2x2 target is in
    // S (with grow, a target joins S while S has room) and whose classical
    // condition fits the condition table.  Counts only when tk is null.
    // Once every qubit carries a left-behind 2x2 gate, no later gate commutes with
    // them all, so the walk stops there (the rest is left behind as a whole).
    std::vector<Cond> conds;
    const uint64_t all_qubits = n >= 64 ? ~0ull : (1ull << n) - 1;
    auto take = [&](uint64_t S0, bool grow, std::vector<POp> *tk, std::vector<POp> *lf, uint64_t *S_out,
                    int *n_u2_out, int *n_ph_out) {
        uint64_t S = S0;
        int cnt = __builtin_popcountll(S0);
        uint64_t ndb = 0, allb = 0;
        int n_u2 = 0, n_ph = 0;
        conds.clear();
        for (auto it = rem.begin(); it != rem.end(); ++it) {
            if (ndb == all_qubits) {
                if (lf) lf->insert(lf->end(), it, rem.end());
                break;
            }
            const POp &p = *it;
            const bool is_u2 = p.op->kind == FusedOp::U2;
            bool ok = (is_u2 ? n_u2 < max_u2 : n_ph < max_ph) && !(p.nd & allb) && !(p.all & ndb);
            if (ok && is_u2) {
                const uint64_t t = 1ull << p.op->q;
                if (!(S & t)) {
                    if (grow && cnt < kTileQubits) {
                        S |= t;
                        ++cnt;
                    } else {
                        ok = false;
                    }
                }
            }
            if (ok && p.op->cond.n) {
                bool found = false;
                for (const auto &cd : conds) found = found || same_cond(cd, p.op->cond);
                if (!found) {
                    if ((int)conds.size() < kTileMaxConds) conds.push_back(p.op->cond);
                    else ok = false;
                }
            }
            if (ok) {
                if (tk) tk->push_back(p);
                if (is_u2) ++n_u2; else ++n_ph;
            } else {
                if (lf) lf->push_back(p);
                ndb |= p.nd;
                allb |= p.all;
            }
        }
        *S_out = S;
        *n_u2_out = n_u2;
        *n_ph_out = n_ph;
    };
    while (!rem.empty()) {
        // ---- choose S and the gates this pass takes: the set that the greedy
        // walk builds, or the contiguous qubits plus a window of consecutive
        // qubits, whichever lets the pass take the most 2x2 gates (then the most
        // gates); a circuit whose gates spread along the qubit line (layers of
        // neighbour couplings) fills passes better with windows
        const uint64_t low = (1ull << kTileContig) - 1;
        uint64_t S = 0, best_S0 = low;
        bool best_grow = true;
        int n_u2 = 0, n_ph = 0;
        take(low, true, nullptr, nullptr, &S, &n_u2, &n_ph);
        int best_u2 = n_u2, best_all = n_u2 + n_ph;
        const int wlen = kTileQubits - kTileContig;
        for (int w = kTileContig; w + wlen <= n; ++w) {
            const uint64_t S0 = low | (((1ull << wlen) - 1) << w);
            uint64_t Sw;
            take(S0, false, nullptr, nullptr, &Sw, &n_u2, &n_ph);
            if (n_u2 > best_u2 || (n_u2 == best_u2 && n_u2 + n_ph > best_all)) {
                best_u2 = n_u2;
                best_all = n_u2 + n_ph;
                best_S0 = S0;
                best_grow = false;
            }
        }
        left.clear();
        taken.clear();
        take(best_S0, best_grow, &taken, &left, &S, &n_u2, &n_ph);
        int cnt = __builtin_popcountll(S);
        // fill S up to 13 qubits with the lowest unused ones
        for (int b = kTileContig; b < n && cnt < kTileQubits; ++b)
            if (!((S >> b) & 1)) {
                S |= 1ull << b;
                ++cnt;
            }

        static thread_local TileParams P;
        std::memset(static_cast<TileHead *>(&P), 0, sizeof(TileHead));
        P.n = n;
        P.n_tiles = 1ull << (n - kTileQubits);
        int local_of[64];
        for (int b = 0; b < 64; ++b) local_of[b] = -1;
        {
            int lb = 0, fb = 0;
            for (int b = 0; b < n; ++b) {
                if ((S >> b) & 1) {
                    P.S[lb] = (int8_t)b;
                    local_of[b] = lb++;
                } else {
                    P.fixed[fb++] = (int8_t)b;
                }
            }
            P.nfix = fb;
            // runs of consecutive fixed qubits
            P.nruns = 0;
            for (int b = 0; b < fb;) {
                int e = b + 1;
                while (e < fb && P.fixed[e] == P.fixed[e - 1] + 1) ++e;
                if (P.nruns >= kTileMaxRuns) {
                    *err = "internal: too many fixed-qubit runs";
                    return QK_EINVAL;
                }
                P.run_tlo[P.nruns] = (uint8_t)b;
                P.run_len[P.nruns] = (uint8_t)(e - b);
                P.run_plo[P.nruns] = (uint8_t)P.fixed[b];
                ++P.nruns;
                b = e;
            }
        }
        P.n_conds = (int)conds.size();
        for (int k = 0; k < P.n_conds; ++k) P.conds[k] = conds[k];

        // ---- list-schedule the taken gates over the arrangements
        const int m = (int)taken.size();
        // dependency edges i -> j (i < j, not commuting) as flat successor lists:
        // the successors of i are succ[succ_at[i] .. succ_at[i + 1])
        static thread_local std::vector<int> npred, succ_at, succ, edge_i, edge_j;
        npred.assign(m, 0);
        succ_at.assign(m + 1, 0);
        edge_i.clear();
        edge_j.clear();
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < j; ++i)
                if (!commute(taken[i], taken[j])) {
                    npred[j]++;
                    succ_at[i + 1]++;
                    edge_i.push_back(i);
                    edge_j.push_back(j);
                }
        for (int i = 0; i < m; ++i) succ_at[i + 1] += succ_at[i];
        succ.resize(edge_i.size());
        {
            static thread_local std::vector<int> fill;
            fill.assign(succ_at.begin(), succ_at.end() - 1);
            for (size_t e = 0; e < edge_i.size(); ++e) succ[fill[edge_i[e]]++] = edge_j[e];   // ascending j per i
        }
        std::vector<char> done(m, 0);
        int ndone = 0, cur = ARR_IO, nops = 0;
        static thread_local std::vector<TileOp> prog;
        prog.assign(2 * (size_t)m + 2, TileOp{});
        auto emit = [&](int j, int arr) {
            const FusedOp &op = *taken[j].op;
            TileOp &t = prog[nops++];
            std::memset(&t, 0, sizeof t);
            t.cond = 0xffff;
            if (op.cond.n)
                for (int k = 0; k < P.n_conds; ++k)
                    if (same_cond(P.conds[k], op.cond)) t.cond = (uint16_t)k;
            if (op.kind == FusedOp::U2) {
                t.kind = TOP_U2;
                int pos;
                slot_of(arr, local_of[op.q], &pos);
                t.k = (uint8_t)pos;
                t.first = (uint16_t)j;   // the FP64 matrix: taken[j]
                encode_cond(op.cmask, op.cmask, arr, local_of, t);
                for (int e = 0; e < 4; ++e) {
                    t.m[2 * e] = (float)op.m[e].real();
                    t.m[2 * e + 1] = (float)op.m[e].imag();
                }
            } else {
                t.kind = TOP_PHASE;
                encode_cond(op.mask, op.val, arr, local_of, t);
                t.ph.re = (float)op.f.real();
                t.ph.im = (float)op.f.imag();
                // the factor's angle as a fraction of a turn in 32-bit fixed point
                double frac = std::arg(op.f) / (2.0 * M_PI);
                if (frac < 0) frac += 1.0;
                t.ph.turns = (uint32_t)(uint64_t)std::llround(frac * 4294967296.0);
            }
            done[j] = 1;
            ++ndone;
            for (int e = succ_at[j]; e < succ_at[j + 1]; ++e) npred[succ[e]]--;
        };
        while (ndone < m) {
            bool progress = false;
            for (int j = 0; j < m; ++j)
                if (!done[j] && npred[j] == 0 && executable(taken[j], cur, local_of)) {
                    emit(j, cur);
                    progress = true;
                }
            if (ndone == m) break;
            if (!progress) {
                int best = -1, best_cnt = -1;
                for (int a = 0; a < 3; ++a) {
                    if (a == cur) continue;
                    int cntr = 0;
                    for (int j = 0; j < m; ++j)
                        if (!done[j] && npred[j] == 0 && executable(taken[j], a, local_of)) ++cntr;
                    if (cntr > best_cnt) {
                        best_cnt = cntr;
                        best = a;
                    }
                }
                TileOp &t = prog[nops++];
                std::memset(&t, 0, sizeof t);
                t.kind = TOP_XPOSE;
                t.k = (uint8_t)best;
                t.cond = 0xffff;
                cur = best;
            }
        }
        if (cur == ARR_LO) {
            TileOp &t = prog[nops++];
            std::memset(&t, 0, sizeof t);
            t.kind = TOP_XPOSE;
            t.k = ARR_IO;
            t.cond = 0xffff;
            cur = ARR_IO;
        }
        // group runs of consecutive diagonal terms by the pending sum they feed
        {
            static thread_local TileOp out[2 * kTileMaxOps + 8];
            int nout = 0, nlin = 0;
            int fixed_index[64];   // physical qubit -> bit of the tile index
            for (int b = 0; b < 64; ++b) fixed_index[b] = -1;
            for (int b = 0; b < P.nfix; ++b) fixed_index[(int)P.fixed[b]] = b;
            bool overflow = false;
            for (int i = 0; i < nops && !overflow;) {
                if (nout >= 2 * kTileMaxOps) {
                    overflow = true;
                    break;
                }
                if (prog[i].kind != TOP_PHASE) {
                    out[nout++] = prog[i++];
                    continue;
                }
                int j = i;
                while (j < nops && prog[j].kind == TOP_PHASE) ++j;
                // per pending sum (register bit 0..4, constant 5): entries that add turns
                struct Term {
                    uint16_t tmask, tval;
                    uint32_t turns;
                    uint64_t gmask, gval;
                };
                std::vector<Term> grp[6];
                // terms on two register bits, reduced to the (1,1) pattern: key -> turns
                struct PairKey {
                    int code;
                    uint16_t tmask, tval;
                    uint64_t gmask, gval;
                    uint32_t turns;
                };
                std::vector<PairKey> pairs;
                auto add_entry = [&](int g, const TileOp &o, uint32_t turns) {
                    Term e;
                    e.tmask = o.tmask;
                    e.tval = o.tval;
                    e.gmask = o.gmask;
                    e.gval = o.gval;
                    e.turns = turns;
                    grp[g].push_back(e);
                };
                for (int t = i; t < j; ++t) {
                    const TileOp &o = prog[t];
                    if (nout >= 2 * kTileMaxOps) {
                        overflow = true;
                        break;
                    }
                    const int pc = __builtin_popcount(o.rmask);
                    const uint32_t T = o.ph.turns;
                    if (o.cond != 0xffff || pc >= 3) {
                        out[nout++] = o;   // applied directly
                        continue;
                    }
                    if (pc == 0) {
                        add_entry(5, o, T);
                    } else if (pc == 1) {
                        const int k = __builtin_ctz(o.rmask);
                        if (o.rval) {
                            add_entry(k, o, T);
                        } else {  // f on bit k = 0:  f * (f^-1 on bit k = 1)
                            add_entry(5, o, T);
                            add_entry(k, o, 0u - T);
                        }
                    } else {
                        // pattern (vk, vl) on register bits k < l as exact sums of a constant,
                        // single-bit terms and a (1,1) pair term
                        const int k = __builtin_ctz(o.rmask), l = 31 - __builtin_clz(o.rmask);
                        const int vk = (o.rval >> k) & 1, vl = (o.rval >> l) & 1;
                        uint32_t pair = T;
                        if (vk && !vl) {
                            add_entry(k, o, T);
                            pair = 0u - T;
                        } else if (!vk && vl) {
                            add_entry(l, o, T);
                            pair = 0u - T;
                        } else if (!vk && !vl) {
                            add_entry(5, o, T);
                            add_entry(k, o, 0u - T);
                            add_entry(l, o, 0u - T);
                        }
                        const int code = k | (l << 3);
                        bool merged = false;
                        for (auto &pk : pairs)
                            if (pk.code == code && pk.tmask == o.tmask && pk.tval == o.tval && pk.gmask == o.gmask &&
                                pk.gval == o.gval) {
                                pk.turns += pair;
                                merged = true;
                                break;
                            }
                        if (!merged) pairs.push_back({code, o.tmask, o.tval, o.gmask, o.gval, pair});
                    }
                }
                for (const auto &pk : pairs) {
                    if (pk.turns == 0) continue;
                    if (nout >= 2 * kTileMaxOps) {
                        overflow = true;
                        break;
                    }
                    TileOp &t = out[nout++];
                    std::memset(&t, 0, sizeof t);
                    t.cond = 0xffff;
                    t.k = (uint8_t)pk.code;
                    if (pk.tmask == 0 && pk.gmask == 0 && pk.turns == 0x80000000u) {
                        t.kind = TOP_PAIRNEG;   // a CZ between two register bits
                        continue;
                    }
                    t.kind = TOP_PAIR;
                    t.rval = 3;   // both bits 1
                    t.tmask = pk.tmask;
                    t.tval = pk.tval;
                    t.gmask = pk.gmask;
                    t.gval = pk.gval;
                    const double ang = 2.0 * M_PI * (double)pk.turns / 4294967296.0;
                    t.ph.re = (float)std::cos(ang);
                    t.ph.im = (float)std::sin(ang);
                    t.ph.turns = pk.turns;
                }
                for (int g = 0; g < 6 && !overflow; ++g) {
                    if (grp[g].empty()) continue;
                    // split the group's terms: the same for every thread and tile
                    // (kept by the planner), and the rest, each a linear term with
                    // its thread-bit and tile-index conditions (TOP_PHASEL)
                    uint32_t host_turns = 0;
                    std::vector<LinTerm> lins;
                    for (const Term &t : grp[g]) {
                        if (t.gmask == 0 && t.tmask == 0) {
                            host_turns += t.turns;
                            continue;
                        }
                        uint32_t fm = 0, fv = 0;   // the fixed-qubit condition on tile-index bits
                        for (uint64_t mk = t.gmask; mk; mk &= mk - 1) {
                            const int pb = __builtin_ctzll(mk), tb = fixed_index[pb];
                            fm |= 1u << tb;
                            if ((t.gval >> pb) & 1) fv |= 1u << tb;
                        }
                        bool merged = false;
                        for (auto &l : lins)
                            if (l.tmask == t.tmask && l.tval == t.tval && l.fmask == fm && l.fval == fv) {
                                l.turns += t.turns;
                                merged = true;
                                break;
                            }
                        if (!merged) {
                            LinTerm l{};
                            l.tmask = t.tmask;
                            l.tval = t.tval;
                            l.fmask = fm;
                            l.fval = fv;
                            l.turns = t.turns;
                            lins.push_back(l);
                        }
                    }
                    if (host_turns != 0) {
                        if (nout >= 2 * kTileMaxOps) { overflow = true; break; }
                        TileOp &t = out[nout++];
                        std::memset(&t, 0, sizeof t);
                        t.kind = TOP_HOSTPH;
                        t.k = (uint8_t)g;
                        t.cond = 0xffff;
                        t.ph.turns = host_turns;
                    }
                    int nl = 0;
                    for (const auto &l : lins) nl += l.turns != 0;
                    if (nl) {
                        if (nout >= 2 * kTileMaxOps || nlin + nl > kTileMaxLin) { overflow = true; break; }
                        TileOp &t = out[nout++];
                        std::memset(&t, 0, sizeof t);
                        t.kind = TOP_PHASEL;
                        t.k = (uint8_t)g;
                        t.cond = 0xffff;
                        t.first = (uint16_t)nlin;
                        for (const auto &l : lins)
                            if (l.turns != 0) P.lin[nlin++] = l;
                        t.count = (uint16_t)(nlin - t.first);
                    }
                }
                i = j;
            }
            if (overflow || nout > kTileMaxOps) {
                // too large for one launch: plan this pass again with fewer gates
                if (max_u2 <= 1 && max_ph <= 1) {
                    *err = "internal: tile program overflow";
                    return QK_EINVAL;
                }
                max_u2 = std::max(1, max_u2 / 2);
                max_ph = std::max(1, max_ph / 2);
                continue;
            }
            // merge runs of consecutive uncontrolled 2x2 gates on distinct
            // register bits into layer ops (they commute with each other)
            int nfin = 0, nmat = 0;
            static thread_local uint16_t lg_mat[kTileMaxMats];   // layer gate -> taken[] index
            for (int i = 0; i < nout && !overflow;) {
                const TileOp &o = out[i];
                const bool plain_u2 = o.kind == TOP_U2 && o.rmask == 0 && o.tmask == 0 && o.gmask == 0 &&
                                      o.cond == 0xffff;
                if (!plain_u2) {
                    if (nfin >= kTileMaxOps) { overflow = true; break; }
                    P.ops[nfin++] = out[i++];
                    continue;
                }
                int bits = 0, j = i;
                while (j < nout) {
                    const TileOp &q = out[j];
                    const bool ok = q.kind == TOP_U2 && q.rmask == 0 && q.tmask == 0 && q.gmask == 0 &&
                                    q.cond == 0xffff && !(bits & (1 << q.k));
                    if (!ok) break;
                    bits |= 1 << q.k;
                    ++j;
                }
                if (nfin >= kTileMaxOps || nmat + (j - i) > kTileMaxMats) { overflow = true; break; }
                TileOp &t = P.ops[nfin++];
                std::memset(&t, 0, sizeof t);
                t.kind = TOP_U2L;
                t.k = (uint8_t)bits;
                t.cond = 0xffff;
                t.first = (uint16_t)nmat;
                t.count = (uint16_t)(j - i);
                // the gates' FP64 matrices in register-bit order; fold_program turns
                // them into pivot coefficients
                for (int b = 0; b < 5; ++b)
                    for (int q = i; q < j; ++q)
                        if (out[q].k == b) lg_mat[nmat++] = out[q].first;
                i = j;
            }
            if (overflow) {
                if (max_u2 <= 1 && max_ph <= 1) {
                    *err = "internal: tile program overflow";
                    return QK_EINVAL;
                }
                max_u2 = std::max(1, max_u2 / 2);
                max_ph = std::max(1, max_ph / 2);
                continue;
            }
            // fold_program: walk the program in order, keeping the pending phases
            // that are the same for every thread (and the scale and the stored bit
            // order of each local qubit) in FP64; layer gates get their pivot
            // coefficients, every other op's conditions are rewritten to the stored
            // order, general gates take their target's uniform phase along to the
            // device, and what is left goes to the final flush
            {
                UniformPending st;
                for (int q = 0; q < kTileQubits; ++q) {
                    st.u[q] = carry[(int)P.S[q]];
                    st.mag[q] = carry_mag[(int)P.S[q]];
                }
                st.u0 = carry_u0;
                st.lam = carry_lam;
                int arr = ARR_IO, w = 0;
                const double pi = M_PI;
                for (int i = 0; i < nfin; ++i) {
                    TileOp o = P.ops[i];
                    // flipped register and thread bits in the current arrangement
                    int rflip = 0, tflip = 0;
                    for (int k = 0; k < 5; ++k) rflip |= st.flip[local_of_reg(arr, k)] << k;
                    for (int t = 0; t < 8; ++t) tflip |= st.flip[local_of_tbit(arr, t)] << t;
                    auto qk_of = [&](int k) { return local_of_reg(arr, k); };
                    switch (o.kind) {
                        case TOP_HOSTPH: {
                            const double ang = turns_angle(o.ph.turns);
                            if (o.k == 5) {
                                st.u0 += ang;
                            } else if (st.flip[qk_of(o.k)]) {  // on the stored |0>
                                st.u0 += ang;
                                st.u[qk_of(o.k)] -= ang;
                            } else {
                                st.u[qk_of(o.k)] += ang;
                            }
                            continue;   // never reaches the device
                        }
                        case TOP_XPOSE:
                            arr = o.k;
                            break;
                        case TOP_U2L: {
                            int idx = o.first;
                            for (int b = 0; b < 5; ++b) {
                                if (!((o.k >> b) & 1)) continue;
                                const FusedOp &fo = *taken[lg_mat[idx]].op;
                                const Mat2 g{{fo.m[0], fo.m[1], fo.m[2], fo.m[3]}};
                                if (pivot_gate(g, st, qk_of(b), P.lg[idx])) o.rmask |= (uint8_t)(1u << b);
                                ++idx;
                            }
                            break;
                        }
                        case TOP_PAIRNEG: {
                            // (-1)^((a^fa)(b^fb)) = (-1)^(ab) (-1)^(fb a) (-1)^(fa b) (-1)^(fa fb)
                            const int ka = o.k & 7, kb = o.k >> 3;
                            const int fa = (rflip >> ka) & 1, fb = (rflip >> kb) & 1;
                            if (fb) st.u[qk_of(ka)] += pi;
                            if (fa) st.u[qk_of(kb)] += pi;
                            if (fa && fb) st.u0 += pi;
                            break;
                        }
                        case TOP_PAIR: {
                            const int ka = o.k & 7, kb = o.k >> 3;
                            const int fa = (rflip >> ka) & 1, fb = (rflip >> kb) & 1;
                            o.tval ^= (uint16_t)(o.tmask & tflip);
                            if (o.tmask == 0 && o.gmask == 0 && o.cond == 0xffff) {
                                // e^{i th} where the true bits a = sa ^ fa, b = sb ^ fb are both
                                // 1, in stored bits: (sa ^ fa)(sb ^ fb) = fa fb + fa (1 - 2 fb) sb
                                // + fb (1 - 2 fa) sa + (1 - 2 fa)(1 - 2 fb) sa sb.  The stored
                                // pattern (1, 1) takes +-th on the device; the constant and the
                                // single-bit parts are uniform phases kept here.
                                const double th = turns_angle(o.ph.turns);
                                if (fa && fb) st.u0 += th;
                                if (fa) st.u[qk_of(kb)] += fb ? -th : th;
                                if (fb) st.u[qk_of(ka)] += fa ? -th : th;
                                if (fa ^ fb) {
                                    o.ph.turns = 0u - o.ph.turns;
                                    o.ph.im = -o.ph.im;
                                }
                                o.rval = 3;
                                o.kind = TOP_PAIRU;
                            } else {
                                o.rval = (uint8_t)(3 ^ (fa | (fb << 1)));
                            }
                            break;
                        }
                        case TOP_PHASEL: {
                            for (int e = o.first; e < o.first + o.count; ++e)
                                P.lin[e].tval ^= (uint16_t)(P.lin[e].tmask & tflip);
                            o.rval = (uint8_t)(o.k < 5 ? (rflip >> o.k) & 1 : 0);
                            // every term tests one bit: "turns where the bit is 1" terms
                            // (TOP_PHASEB), a term on a bit being 0 split into a
                            // constant kept here and a negated bit-1 term
                            bool single = true;
                            for (int e = o.first; e < o.first + o.count; ++e)
                                single = single && __builtin_popcount(P.lin[e].tmask) + __builtin_popcount(P.lin[e].fmask) == 1;
                            if (!single) break;
                            std::vector<BitTerm> th, ti;
                            uint32_t cst = 0;
                            for (int e = o.first; e < o.first + o.count; ++e) {
                                const LinTerm &L = P.lin[e];
                                const bool thread = L.tmask != 0;
                                const uint32_t b = thread ? (uint32_t)__builtin_ctz(L.tmask) : (uint32_t)__builtin_ctz(L.fmask);
                                const uint32_t v = thread ? ((uint32_t)L.tval >> b) & 1u : (L.fval >> b) & 1u;
                                uint32_t t = L.turns;
                                if (!v) {
                                    cst += t;
                                    t = 0u - t;
                                }
                                (thread ? th : ti).push_back(BitTerm{b, t});
                            }
                            BitTerm *bt = reinterpret_cast<BitTerm *>(&P.lin[o.first]);
                            for (size_t q = 0; q < th.size(); ++q) bt[q] = th[q];
                            for (size_t q = 0; q < ti.size(); ++q) bt[th.size() + q] = ti[q];
                            o.kind = TOP_PHASEB;
                            o.first = (uint16_t)(2 * o.first);
                            o.count = (uint16_t)th.size();
                            o.count2 = (uint16_t)ti.size();
                            if (cst) {   // the same for every thread and tile: kept here
                                const double ang = turns_angle(cst);
                                if (o.k == 5) {
                                    st.u0 += ang;
                                } else if (st.flip[qk_of(o.k)]) {
                                    st.u0 += ang;
                                    st.u[qk_of(o.k)] -= ang;
                                } else {
                                    st.u[qk_of(o.k)] += ang;
                                }
                            }
                            break;
                        }
                        case TOP_PHASE:
                            o.rval ^= (uint8_t)(o.rmask & rflip);
                            o.tval ^= (uint16_t)(o.tmask & tflip);
                            break;
                        case TOP_U2: {
                            const int q = qk_of(o.k);
                            o.rval ^= (uint8_t)(o.rmask & rflip);
                            o.tval ^= (uint16_t)(o.tmask & tflip);
                            if (st.flip[q]) {  // X U X in stored order
                                float t[8];
                                std::memcpy(t, o.m, sizeof t);
                                const int perm[4] = {3, 2, 1, 0};
                                for (int e = 0; e < 4; ++e) {
                                    o.m[2 * e] = t[2 * perm[e]];
                                    o.m[2 * e + 1] = t[2 * perm[e] + 1];
                                }
                            }
                            o.hturns = angle_turns(st.u[q]);
                            o.hmag = (float)st.mag[q];
                            st.u[q] = 0.0;
                            st.mag[q] = 1.0;
                            break;
                        }
                        default:
                            break;
                    }
                    P.ops[w++] = o;
                }
                nfin = w;
                // a CZ between register bits right after a layer op (nothing between
                // them) becomes a bit of that op's CZ mask: one dispatch fewer
                w = 0;
                for (int i = 0; i < nfin; ++i) {
                    const TileOp &o = P.ops[i];
                    if (o.kind == TOP_PAIRNEG && w > 0 && P.ops[w - 1].kind == TOP_U2L) {
                        P.ops[w - 1].tmask |= (uint16_t)(1u << cz_index(o.k & 7, o.k >> 3));
                        continue;
                    }
                    P.ops[w++] = o;
                }
                nfin = w;
                P.fin_flip = 0;
                for (int q = 0; q < kTileQubits; ++q) P.fin_flip |= st.flip[q] << q;
                P.fin_fixed_mask = 0;
                if (left.empty()) {   // the plan's last pass applies everything pending
                    for (int q = 0; q < kTileQubits; ++q) {
                        P.fin_turns[q] = angle_turns(st.u[q]);
                        P.fin_mag[q] = (float)st.mag[q];
                    }
                    P.fin_turns[13] = angle_turns(st.u0);
                    P.fin_scale = (float)st.lam;
                    for (int b = 0; b < P.nfix; ++b) {
                        const uint32_t t = angle_turns(carry[(int)P.fixed[b]]);
                        P.fin_fixed[b] = t;
                        P.fin_fixed_mag[b] = (float)carry_mag[(int)P.fixed[b]];
                        if (t || P.fin_fixed_mag[b] != 1.f) P.fin_fixed_mask |= 1ull << b;
                    }
                } else {              // hand the uniform part to the next pass
                    for (int q = 0; q < kTileQubits; ++q) {
                        // a qubit stored flipped has its factor F on |0>: F on |0> is F
                        // overall times 1 / F on |1>
                        const int pq = (int)P.S[q];
                        if (st.flip[q]) {
                            carry[pq] = -st.u[q];
                            carry_mag[pq] = 1.0 / st.mag[q];
                            st.u0 += st.u[q];
                            st.lam *= st.mag[q];
                        } else {
                            carry[pq] = st.u[q];
                            carry_mag[pq] = st.mag[q];
                        }
                        P.fin_turns[q] = 0;
                        P.fin_mag[q] = 1.f;
                    }
                    carry_u0 = st.u0;
                    P.fin_turns[13] = 0;
                    // the stored amplitudes are the true ones divided by the scale
                    // (a factor in [2^-1/2, 2] per gate): keep them within 2^24 of it
                    // in FP32
                    if (st.lam < 0x1p-24 || st.lam > 0x1p24) {
                        P.fin_scale = (float)st.lam;
                        carry_lam = 1.0;
                    } else {
                        P.fin_scale = 1.f;
                        carry_lam = st.lam;
                    }
                }
            }
            nops = nfin;
            P.nlg = nmat;
            P.nlin = nlin;
            // whether any phase factor the pass forms can be other than 1 or -1 (the
            // kernel fills its phase table only then)
            {
                auto general = [](uint32_t t) { return t != 0u && t != 0x80000000u; };
                bool need = false;
                for (int i = 0; i < nops && !need; ++i) {
                    const TileOp &o = P.ops[i];
                    if (o.kind == TOP_U2 || o.kind == TOP_PHASE) need = true;
                    if (o.kind == TOP_PHASEL)
                        for (int e = o.first; e < o.first + o.count; ++e) need = need || general(P.lin[e].turns);
                    if (o.kind == TOP_PHASEB) {
                        const BitTerm *bt = reinterpret_cast<const BitTerm *>(&P.lin[0]) + o.first;
                        for (int e = 0; e < o.count + o.count2; ++e) need = need || general(bt[e].turns);
                    }
                }
                for (int q = 0; q < 14; ++q) need = need || general(P.fin_turns[q]);
                for (int b = 0; b < P.nfix; ++b)
                    if ((P.fin_fixed_mask >> b) & 1) need = need || general(P.fin_fixed[b]);
                P.need_tab = need ? 1 : 0;
            }
        }
        P.nops = nops;
        P.store_arr = cur;
        if (planner->log) {
            int cnt_k[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // by TileOpKind
            for (int i = 0; i < nops; ++i) cnt_k[P.ops[i].kind]++;
            std::fprintf(stderr,
                         "[qk plan] pass S=%#llx gates=%d (u2 %d, phase %d) ops=%d u2=%d layers=%d phase_direct=%d "
                         "phase_groups=%d terms=%d pairs=%d pair_signs=%d xpose=%d store_arr=%d\n",
                         (unsigned long long)S, m, n_u2, n_ph, nops, cnt_k[TOP_U2], cnt_k[TOP_U2L], cnt_k[TOP_PHASE],
                         cnt_k[TOP_PHASEL], P.nlin, cnt_k[TOP_PAIR], cnt_k[TOP_PAIRNEG], cnt_k[TOP_XPOSE], cur);
        }

        const qk_status st = sink(P);
        if (st != QK_OK) return st;
        rem.swap(left);
        max_u2 = 100;
        max_ph = 300;
    }
    return QK_OK;
}

qk_status run_fused(TilePlanner *planner, qk_ctx *c, const std::vector<FusedOp> &ops) {
    const int n = ctx_n(c);
    if (n < kTileQubits || ctx_prec(c) != 0) {
        for (const auto &op : ops) {
            qk_status s = ctx_run_plain(c, op);
            if (s != QK_OK) return s;
        }
        return QK_OK;
    }
    const PassSink launch = [&](TileParams &P) -> qk_status {
        void *tok = nullptr;
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        if (planner->log) {  // trace mode: time this pass on its own (synchronous)
            cudaEventCreate(&ev0);
            cudaEventCreate(&ev1);
            cudaEventRecord(ev0, ctx_stream(c));
        }
        ctx_launch_begin(c, 0, 2.0 * 8.0 * (double)(1ull << n), &tok);
        cudaError_t e = launch_tile(ctx_state(c), P, ctx_cbits(c), ctx_stream(c));
        ctx_launch_end(tok);
        if (e != cudaSuccess) return ctx_fail(c, QK_ECUDA, cudaGetErrorString(e));
        if (planner->log) {
            float ms = 0.f;
            cudaEventRecord(ev1, ctx_stream(c));
            cudaEventSynchronize(ev1);
            cudaEventElapsedTime(&ms, ev0, ev1);
            std::fprintf(stderr, "[qk plan]   %.3f ms\n", ms);
            cudaEventDestroy(ev0);
            cudaEventDestroy(ev1);
        }
        return QK_OK;
    };
    const char *err = "";
    const qk_status st = plan_passes(planner, n, ops, launch, &err);
    if (st != QK_OK && err[0]) return ctx_fail(c, st, err);
    return st;
}

}  // namespace qk
