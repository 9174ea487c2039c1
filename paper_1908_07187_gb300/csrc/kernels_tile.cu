// K3: fused tile pass for complex64 states.
//
// One CTA owns one tile of 2^13 amplitudes (13 physical qubits S[0..12]; the
// other n-13 bits are fixed by the tile index).  The tile is read from HBM once,
// a program of gates runs on it, and it is written back once, so a pass costs
// one read + one write of the state however many gates it carries.
//
// Each of the 256 threads holds 32 amplitudes in registers, split into real and
// imaginary parts, two amplitudes per float2 (re[2j], re[2j+1]) /
// (im[2j], im[2j+1]), so that a butterfly on register bit K >= 1 runs as packed
// f32x2 FMAs on two amplitude pairs at once.  The register bits are changed by
// transposing the tile through shared memory (three fixed arrangements, see
// qk_kernels.cuh).
//
// Uncontrolled gates run in pivot form (LayerGate in qk_kernels.cuh): 8 FP32
// FMAs per amplitude pair (in place) instead of the 16 operations of a complex
// 2x2 product.  What the pivot form leaves over -- a real scale, the same for
// every amplitude of the pass, and per-qubit factors -- stays pending.  The parts
// that are the same for every thread are tracked by the planner and folded into
// later gates' coefficients or the final flush; each thread only keeps the parts
// that depend on its own bits
// (diagonal terms coupling a register bit with a lane, warp or fixed bit), as six
// 32-bit fixed-point phase sums (exact modulo one turn): one per register bit
// and one for the whole thread.  A sum of exactly half a turn is a sign flip and
// costs no phase factor.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>

#include "qk_kernels.cuh"

namespace qk {
namespace {

constexpr uint32_t kHalfTurn = 0x80000000u;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 splat(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float xor_sign(float x, uint32_t s) { return __uint_as_float(__float_as_uint(x) ^ s); }

// exp(2 pi i j / 256) for j < 256, filled once per CTA
__shared__ float2 s_turn_tab[256];

__device__ __forceinline__ void fill_turn_table() {
    for (int j = threadIdx.x; j < 256; j += blockDim.x) {
        float s, c;
        sincospif((float)j * (1.f / 128.f), &s, &c);
        s_turn_tab[j] = make_float2(c, s);
    }
}

// exp(2 pi i t / 2^32): the table entry of the top 8 bits times the short
// Taylor series of the remaining angle x = 2 pi (t mod 2^24) / 2^32 < 2 pi / 256
// (cos x = 1 - x^2/2 + x^4/24, sin x = x - x^3/6; the next terms are below
// 2^-30), about a dozen FP32 operations instead of a full sincos.
__device__ __forceinline__ float2 turns_to_phase(uint32_t t) {
    const float2 a = s_turn_tab[t >> 24];
    const float x = (float)(t & 0xFFFFFFu) * 1.46291807926715968e-9f;  // 2 pi / 2^32
    const float x2 = x * x;
    const float c = fmaf(x2, fmaf(x2, 1.f / 24.f, -0.5f), 1.f);
    const float s = x * fmaf(x2, -1.f / 6.f, 1.f);
    return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
}
// the same, exact for the sign flips that CZ-type terms produce
__device__ __forceinline__ float2 phase_of(uint32_t t) {
    if (t == 0u) return make_float2(1.f, 0.f);
    if (t == kHalfTurn) return make_float2(-1.f, 0.f);
    return turns_to_phase(t);
}

// Amplitudes of one thread: R[j] = (re[2j], re[2j+1]), I[j] = (im[2j], im[2j+1]).
struct Regs {
    float2 R[16], I[16];
};

template <int r>
__device__ __forceinline__ float &re_of(Regs &v) {
    if constexpr (r & 1) return v.R[r >> 1].y;
    else return v.R[r >> 1].x;
}
template <int r>
__device__ __forceinline__ float &im_of(Regs &v) {
    if constexpr (r & 1) return v.I[r >> 1].y;
    else return v.I[r >> 1].x;
}

// Thread-dependent pending phases: t(k) on register bit k = 1, t0 on the whole
// thread.  The sums live in shared memory (word w of thread x at w * kTileThreads
// + x, conflict-free), leaving the registers to the amplitudes; a register mask
// says which sums may be nonzero, so a thread with nothing pending touches no
// shared memory.
struct DevPending {
    uint32_t *p;   // word 0: t0, word 1 + k: t(k)
    int mask;      // bit k: t(k) may be nonzero; bit 5: t0 may be nonzero
    __device__ __forceinline__ uint32_t &w(int k) { return p[(k + 1) * kTileThreads]; }  // k = -1: t0
    __device__ __forceinline__ void reset() { mask = 0; }
    __device__ __forceinline__ uint32_t get(int k) { return (mask >> k) & 1 ? w(k) : 0u; }
    __device__ __forceinline__ uint32_t get0() { return mask & 32 ? w(-1) : 0u; }
    __device__ __forceinline__ void set(int k, uint32_t x) {
        w(k) = x;
        mask |= 1 << k;
    }
    __device__ __forceinline__ void set0(uint32_t x) {
        w(-1) = x;
        mask |= 32;
    }
    __device__ __forceinline__ void add(int k, uint32_t d) {  // k == 5: t0
        if (k == 5) set0(get0() + d);
        else set(k, get(k) + d);
    }
    __device__ __forceinline__ void clear(int k) { mask &= ~(1 << k); }
};

// Shared-memory slot (in floats, separate real and imaginary planes) of local
// index L.  The map is linear over GF(2), so slot(thread part ^ register part)
// = slot(thread part) ^ slot(register part), and every arrangement's warp access
// touches 32 distinct banks.
__host__ __device__ constexpr int slot4(int L) { return L ^ (((L >> 5) ^ (L >> 10)) & 31); }

template <int ARR>
__host__ __device__ constexpr int reg_part(int r) {
    return ARR == ARR_IO ? (r << 5) : ARR == ARR_LO ? r : (r << 8);
}
template <int ARR>
__device__ __forceinline__ int thread_part(int lane, int warp) {
    if constexpr (ARR == ARR_IO) return lane | (warp << 10);
    else if constexpr (ARR == ARR_LO) return (lane << 5) | (warp << 10);
    else return lane | (warp << 5);
}

template <int ARR, int r>
__device__ __forceinline__ void put_one(float *sre, float *sim, Regs &v, int tslot) {
    constexpr int rs = slot4(reg_part<ARR>(r));
    sre[tslot ^ rs] = re_of<r>(v);
    sim[tslot ^ rs] = im_of<r>(v);
}
template <int ARR, int r>
__device__ __forceinline__ void get_one(const float *sre, const float *sim, Regs &v, int tslot) {
    constexpr int rs = slot4(reg_part<ARR>(r));
    re_of<r>(v) = sre[tslot ^ rs];
    im_of<r>(v) = sim[tslot ^ rs];
}

template <int ARR, int... rs>
__device__ __forceinline__ void put_all(float *sre, float *sim, Regs &v, int tslot, std::integer_sequence<int, rs...>) {
    (put_one<ARR, rs>(sre, sim, v, tslot), ...);
}
template <int ARR, int... rs>
__device__ __forceinline__ void get_all(const float *sre, const float *sim, Regs &v, int tslot,
                                        std::integer_sequence<int, rs...>) {
    (get_one<ARR, rs>(sre, sim, v, tslot), ...);
}

template <int ARR>
__device__ __forceinline__ void to_smem(float *sre, float *sim, Regs &v, int lane, int warp) {
    put_all<ARR>(sre, sim, v, slot4(thread_part<ARR>(lane, warp)), std::make_integer_sequence<int, 32>{});
}
template <int ARR>
__device__ __forceinline__ void from_smem(const float *sre, const float *sim, Regs &v, int lane, int warp) {
    get_all<ARR>(sre, sim, v, slot4(thread_part<ARR>(lane, warp)), std::make_integer_sequence<int, 32>{});
}

__device__ __forceinline__ void transpose(Regs &v, float *sre, float *sim, int from, int to, int lane, int warp) {
    __syncthreads();
    if (from == ARR_IO) to_smem<ARR_IO>(sre, sim, v, lane, warp);
    else if (from == ARR_LO) to_smem<ARR_LO>(sre, sim, v, lane, warp);
    else to_smem<ARR_HI>(sre, sim, v, lane, warp);
    __syncthreads();
    if (to == ARR_IO) from_smem<ARR_IO>(sre, sim, v, lane, warp);
    else if (to == ARR_LO) from_smem<ARR_LO>(sre, sim, v, lane, warp);
    else from_smem<ARR_HI>(sre, sim, v, lane, warp);
}

// ---------------------------------------------------------------------------
// pending-phase flushes
// ---------------------------------------------------------------------------

// Every sum is 0 or half a turn: amplitude r changes sign iff t0 + sum_k r_k t_k
// is half a turn (sign bits combined by XOR, applied to the float sign bits).
__device__ __forceinline__ void flush_signs(Regs &v, uint32_t t0, const uint32_t t[5]) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        uint32_t s = t0;
        if (j & 1) s ^= t[1];
        if (j & 2) s ^= t[2];
        if (j & 4) s ^= t[3];
        if (j & 8) s ^= t[4];
        const uint32_t so = s ^ t[0];
        v.R[j].x = xor_sign(v.R[j].x, s);
        v.I[j].x = xor_sign(v.I[j].x, s);
        v.R[j].y = xor_sign(v.R[j].y, so);
        v.I[j].y = xor_sign(v.I[j].y, so);
    }
}

// General diagonal D(r) = c0 * prod_{k in r} a_k on the 32 registers (any
// magnitudes): per value of register bits 1, 2 the factor q = c0 a1^r1 a2^r2,
// then per value of bits 3, 4 one more product, and one for register bit 0.
__device__ __forceinline__ void apply_diagonal(Regs &v, float2 c0, const float2 a[5]) {
    const float2 a12 = cmul(a[1], a[2]), a34 = cmul(a[3], a[4]);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const float2 q = l == 0 ? c0 : cmul(c0, l == 1 ? a[1] : l == 2 ? a[2] : a12);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int j = 4 * h + l;   // float2 j: register bits 1, 2 = l, bits 3, 4 = h
            const float2 D = h == 0 ? q : cmul(q, h == 1 ? a[3] : h == 2 ? a[4] : a34);
            const float2 d1 = cmul(D, a[0]);
            const float2 Dr = make_float2(D.x, d1.x), Di = make_float2(D.y, d1.y);
            const float2 A = v.R[j], B = v.I[j];
            v.R[j] = ffma2(neg2(Di), B, __fmul2_rn(Dr, A));
            v.I[j] = ffma2(Di, A, __fmul2_rn(Dr, B));
        }
    }
}

// amplitudes with register bit K set are multiplied by f
template <int K>
__device__ __forceinline__ void bit_factor(Regs &v, float2 f) {
    if constexpr (K == 0) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float xr = v.R[j].y, xi = v.I[j].y;
            v.R[j].y = xr * f.x - xi * f.y;
            v.I[j].y = xr * f.y + xi * f.x;
        }
    } else {
        const float2 fr = splat(f.x), fi = splat(f.y), nfi = splat(-f.y);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (!(j & (1 << (K - 1)))) continue;
            const float2 A = v.R[j], B = v.I[j];
            v.R[j] = ffma2(nfi, B, __fmul2_rn(fr, A));
            v.I[j] = ffma2(fi, A, __fmul2_rn(fr, B));
        }
    }
}

__device__ __forceinline__ void bit_factor_dispatch(int k, Regs &v, float2 f) {
    switch (k) {
        case 0: bit_factor<0>(v, f); break;
        case 1: bit_factor<1>(v, f); break;
        case 2: bit_factor<2>(v, f); break;
        case 3: bit_factor<3>(v, f); break;
        default: bit_factor<4>(v, f); break;
    }
}

// Materialise the thread's pending phases (before a transpose moves amplitudes
// between threads).
__device__ __forceinline__ void flush_dev(Regs &v, DevPending &pd) {
    if (pd.mask == 0) return;
    uint32_t t[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) t[k] = pd.get(k);
    const uint32_t t0 = pd.get0();
    if (((t[0] | t[1] | t[2] | t[3] | t[4] | t0) & ~kHalfTurn) == 0u) {
        flush_signs(v, t0, t);
    } else {
        float2 a[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) a[k] = phase_of(t[k]);
        apply_diagonal(v, phase_of(t0), a);
    }
    pd.reset();
}

// ---------------------------------------------------------------------------
// gates
// ---------------------------------------------------------------------------

// Pivot butterfly on register bit K >= 1 (see LayerGate): couples float2
// registers (j, j | 2^(K-1)), two amplitude pairs per couple, in place in the
// amplitudes' own registers.  ZF = 0: y1 += c1 y0, then y0 += c0 y1 with the new
// y1; ZF = 1: y0 += c0 y1, then y1 += c1 y0 with the new y0.  8 packed FMAs per
// couple.
template <int K, int ZF>
__device__ __forceinline__ void piv_packed(Regs &v, float2 c0r, float2 c0i, float2 nc0i, float2 c1r, float2 c1i,
                                           float2 nc1i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (j & (1 << (K - 1))) continue;
        const int j1 = j | (1 << (K - 1));
        float2 A = v.R[j], B = v.I[j], C = v.R[j1], D = v.I[j1];
        if constexpr (ZF == 0) {
            C = ffma2(nc1i, B, ffma2(c1r, A, C));
            D = ffma2(c1i, A, ffma2(c1r, B, D));
            A = ffma2(nc0i, D, ffma2(c0r, C, A));
            B = ffma2(c0i, C, ffma2(c0r, D, B));
        } else {
            A = ffma2(nc0i, D, ffma2(c0r, C, A));
            B = ffma2(c0i, C, ffma2(c0r, D, B));
            C = ffma2(nc1i, B, ffma2(c1r, A, C));
            D = ffma2(c1i, A, ffma2(c1r, B, D));
        }
        v.R[j] = A;
        v.I[j] = B;
        v.R[j1] = C;
        v.I[j1] = D;
    }
}

// Pivot butterfly on register bit 0: the pair is the two halves of one float2.
template <int ZF>
__device__ __forceinline__ void piv_bit0(Regs &v, float c0r, float c0i, float c1r, float c1i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        float y0r = v.R[j].x, y0i = v.I[j].x, y1r = v.R[j].y, y1i = v.I[j].y;
        if constexpr (ZF == 0) {
            y1r = fmaf(-c1i, y0i, fmaf(c1r, y0r, y1r));
            y1i = fmaf(c1i, y0r, fmaf(c1r, y0i, y1i));
            y0r = fmaf(-c0i, y1i, fmaf(c0r, y1r, y0r));
            y0i = fmaf(c0i, y1r, fmaf(c0r, y1i, y0i));
        } else {
            y0r = fmaf(-c0i, y1i, fmaf(c0r, y1r, y0r));
            y0i = fmaf(c0i, y1r, fmaf(c0r, y1i, y0i));
            y1r = fmaf(-c1i, y0i, fmaf(c1r, y0r, y1r));
            y1i = fmaf(c1i, y0r, fmaf(c1r, y0i, y1i));
        }
        v.R[j] = make_float2(y0r, y1r);
        v.I[j] = make_float2(y0i, y1i);
    }
}

// One gate of a TOP_U2L layer on register bit K.  The planner folded every
// pending factor that is the same for all threads into its coefficients C0, C1
// and chose the stored bit order so that the pivot is the diagonal entry; the
// thread's own pending phase e of bit K turns them into c0 = C0 e and
// c1 = C1 conj(e), and leaves e pending on the bit.  zf: which value of the pair
// is updated first (see LayerGate).
template <int K>
__device__ __forceinline__ void layer_gate(Regs &v, DevPending &pd, const LayerGate &g, bool zf) {
    float2 a0r = g.c[0], a0i = g.c[1], na0i = g.c[2], a1r = g.c[3], a1i = g.c[4], na1i = g.c[5];
    const uint32_t tk = pd.get(K);
    if (tk != 0u) {
        if (tk == kHalfTurn) {
            a0r = neg2(a0r); a0i = neg2(a0i); na0i = neg2(na0i);
            a1r = neg2(a1r); a1i = neg2(a1i); na1i = neg2(na1i);
        } else {
            const float2 e = turns_to_phase(tk);
            const float2 x0 = cmul(make_float2(a0r.x, a0i.x), e);
            const float2 x1 = cmul(make_float2(a1r.x, a1i.x), conj2(e));
            a0r = splat(x0.x); a0i = splat(x0.y); na0i = splat(-x0.y);
            a1r = splat(x1.x); a1i = splat(x1.y); na1i = splat(-x1.y);
        }
    }
    if constexpr (K == 0) {
        if (zf) piv_bit0<1>(v, a0r.x, a0i.x, a1r.x, a1i.x);
        else piv_bit0<0>(v, a0r.x, a0i.x, a1r.x, a1i.x);
    } else {
        if (zf) piv_packed<K, 1>(v, a0r, a0i, na0i, a1r, a1i, na1i);
        else piv_packed<K, 0>(v, a0r, a0i, na0i, a1r, a1i, na1i);
    }
}

// General 2x2 gate on register bit K >= 1 where the register bits in rmask are 1
// (a controlled gate with register-bit controls); with register bit 0 in rmask
// only the odd halves act.  Scalar FMAs keep the coefficients to eight registers.
__device__ __forceinline__ float2 mv2(float2 m0, float2 x0, float2 m1, float2 x1) {  // m0 x0 + m1 x1
    return make_float2(fmaf(-m1.y, x1.y, fmaf(m1.x, x1.x, fmaf(-m0.y, x0.y, m0.x * x0.x))),
                       fmaf(m1.y, x1.x, fmaf(m1.x, x1.y, fmaf(m0.y, x0.x, m0.x * x0.y))));
}
template <int K>
__device__ __forceinline__ void u2_packed(Regs &v, float2 m00, float2 m01, float2 m10, float2 m11, int rmask,
                                          int rval) {
    static_assert(K >= 1 && K <= 4, "K >= 1");
    // register bit 0 in rmask: only the halves with that bit value act
    const bool act_x = !(rmask & 1) || !(rval & 1), act_y = !(rmask & 1) || (rval & 1);
    const int hmask = rmask & ~1, hval = rval & ~1;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (j & (1 << (K - 1))) continue;
        const int j1 = j | (1 << (K - 1));
        if (((j << 1) & hmask) != hval) continue;
        // two amplitude pairs: (.x halves) and (.y halves)
        const float2 a0 = make_float2(v.R[j].x, v.I[j].x), b0 = make_float2(v.R[j1].x, v.I[j1].x);
        const float2 a1 = make_float2(v.R[j].y, v.I[j].y), b1 = make_float2(v.R[j1].y, v.I[j1].y);
        if (act_y) {
            const float2 o1 = mv2(m00, a1, m01, b1), p1 = mv2(m10, a1, m11, b1);
            v.R[j].y = o1.x; v.I[j].y = o1.y; v.R[j1].y = p1.x; v.I[j1].y = p1.y;
        }
        if (act_x) {
            const float2 o0 = mv2(m00, a0, m01, b0), p0 = mv2(m10, a0, m11, b0);
            v.R[j].x = o0.x; v.I[j].x = o0.y; v.R[j1].x = p0.x; v.I[j1].x = p0.y;
        }
    }
}

// General 2x2 gate on register bit 0: the pair is the two halves of one float2.
__device__ __forceinline__ void u2_bit0(Regs &v, float2 m00, float2 m01, float2 m10, float2 m11, int rmask,
                                        int rval) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (((j << 1) & rmask) != rval) continue;
        const float2 a = make_float2(v.R[j].x, v.I[j].x), b = make_float2(v.R[j].y, v.I[j].y);
        const float2 o0 = make_float2(m00.x * a.x - m00.y * a.y + m01.x * b.x - m01.y * b.y,
                                      m00.x * a.y + m00.y * a.x + m01.x * b.y + m01.y * b.x);
        const float2 o1 = make_float2(m10.x * a.x - m10.y * a.y + m11.x * b.x - m11.y * b.y,
                                      m10.x * a.y + m10.y * a.x + m11.x * b.y + m11.y * b.x);
        v.R[j] = make_float2(o0.x, o1.x);
        v.I[j] = make_float2(o0.y, o1.y);
    }
}

// amplitudes whose register bits K < L have the values PAT (bit 0: K, bit 1: L)
// are multiplied by f.  With K >= 1 the affected amplitudes fill whole float2
// registers (register bit 0 is free), four of R and four of I: packed products.
template <int K, int L, int PAT, int r>
__device__ __forceinline__ void pair_one(Regs &v, float2 f) {
    constexpr int rp = ((r >> K) & 1) | (((r >> L) & 1) << 1);
    if constexpr (rp == PAT) {
        float &x = re_of<r>(v);
        float &y = im_of<r>(v);
        const float xr = x, xi = y;
        x = xr * f.x - xi * f.y;
        y = xr * f.y + xi * f.x;
    }
}
template <int K, int L, int PAT, int... rs>
__device__ __forceinline__ void pair_all(Regs &v, float2 f, std::integer_sequence<int, rs...>) {
    (pair_one<K, L, PAT, rs>(v, f), ...);
}
template <int K, int L, int PAT>
__device__ __forceinline__ void pair_pat(Regs &v, float2 f) {
    if constexpr (K >= 1) {
        const float2 fr = splat(f.x), fi = splat(f.y), nfi = splat(-f.y);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int rp = ((j >> (K - 1)) & 1) | (((j >> (L - 1)) & 1) << 1);
            if (rp != PAT) continue;
            const float2 A = v.R[j], B = v.I[j];
            v.R[j] = ffma2(nfi, B, __fmul2_rn(fr, A));
            v.I[j] = ffma2(fi, A, __fmul2_rn(fr, B));
        }
    } else {
        pair_all<K, L, PAT>(v, f, std::make_integer_sequence<int, 32>{});
    }
}
template <int K, int L>
__device__ __forceinline__ void pair_factor(Regs &v, float2 f, int pat) {
    switch (pat) {
        case 0: pair_pat<K, L, 0>(v, f); break;
        case 1: pair_pat<K, L, 1>(v, f); break;
        case 2: pair_pat<K, L, 2>(v, f); break;
        default: pair_pat<K, L, 3>(v, f); break;
    }
}

template <int K, int L, int r>
__device__ __forceinline__ void pair_neg_one(Regs &v) {
    if constexpr (((r >> K) & 1) && ((r >> L) & 1)) {
        re_of<r>(v) = -re_of<r>(v);
        im_of<r>(v) = -im_of<r>(v);
    }
}
template <int K, int L, int... rs>
__device__ __forceinline__ void pair_neg_all(Regs &v, std::integer_sequence<int, rs...>) {
    (pair_neg_one<K, L, rs>(v), ...);
}
// the CZs of a layer op's mask (bit cz_index(k, l) for the pair k < l)
__device__ __forceinline__ void cz_mask(Regs &v, int m) {
    constexpr auto seq = std::make_integer_sequence<int, 32>{};
    if (m & (1 << cz_index(0, 1))) pair_neg_all<0, 1>(v, seq);
    if (m & (1 << cz_index(0, 2))) pair_neg_all<0, 2>(v, seq);
    if (m & (1 << cz_index(0, 3))) pair_neg_all<0, 3>(v, seq);
    if (m & (1 << cz_index(0, 4))) pair_neg_all<0, 4>(v, seq);
    if (m & (1 << cz_index(1, 2))) pair_neg_all<1, 2>(v, seq);
    if (m & (1 << cz_index(1, 3))) pair_neg_all<1, 3>(v, seq);
    if (m & (1 << cz_index(1, 4))) pair_neg_all<1, 4>(v, seq);
    if (m & (1 << cz_index(2, 3))) pair_neg_all<2, 3>(v, seq);
    if (m & (1 << cz_index(2, 4))) pair_neg_all<2, 4>(v, seq);
    if (m & (1 << cz_index(3, 4))) pair_neg_all<3, 4>(v, seq);
}

// sign flip of the amplitudes whose register bits k and l are both 1 (code k | l << 3)
__device__ __forceinline__ void pair_neg(Regs &v, int code) {
    constexpr auto seq = std::make_integer_sequence<int, 32>{};
    switch (code) {
        case 0 | (1 << 3): pair_neg_all<0, 1>(v, seq); break;
        case 0 | (2 << 3): pair_neg_all<0, 2>(v, seq); break;
        case 0 | (3 << 3): pair_neg_all<0, 3>(v, seq); break;
        case 0 | (4 << 3): pair_neg_all<0, 4>(v, seq); break;
        case 1 | (2 << 3): pair_neg_all<1, 2>(v, seq); break;
        case 1 | (3 << 3): pair_neg_all<1, 3>(v, seq); break;
        case 1 | (4 << 3): pair_neg_all<1, 4>(v, seq); break;
        case 2 | (3 << 3): pair_neg_all<2, 3>(v, seq); break;
        case 2 | (4 << 3): pair_neg_all<2, 4>(v, seq); break;
        default: pair_neg_all<3, 4>(v, seq); break;
    }
}

// pair factor on register bits (code k | l << 3), pattern pat of the two bits
__device__ __forceinline__ void pair_dispatch(Regs &v, int code, float2 f, int pat) {
    switch (code) {
        case 0 | (1 << 3): pair_factor<0, 1>(v, f, pat); break;
        case 0 | (2 << 3): pair_factor<0, 2>(v, f, pat); break;
        case 0 | (3 << 3): pair_factor<0, 3>(v, f, pat); break;
        case 0 | (4 << 3): pair_factor<0, 4>(v, f, pat); break;
        case 1 | (2 << 3): pair_factor<1, 2>(v, f, pat); break;
        case 1 | (3 << 3): pair_factor<1, 3>(v, f, pat); break;
        case 1 | (4 << 3): pair_factor<1, 4>(v, f, pat); break;
        case 2 | (3 << 3): pair_factor<2, 3>(v, f, pat); break;
        case 2 | (4 << 3): pair_factor<2, 4>(v, f, pat); break;
        default: pair_factor<3, 4>(v, f, pat); break;
    }
}

// TOP_PAIRU: the pattern is always (1, 1) (the planner moves the other patterns'
// constant and single-bit parts into its uniform phases)
__device__ __forceinline__ void pair11_dispatch(Regs &v, int code, float2 f) {
    switch (code) {
        case 0 | (1 << 3): pair_pat<0, 1, 3>(v, f); break;
        case 0 | (2 << 3): pair_pat<0, 2, 3>(v, f); break;
        case 0 | (3 << 3): pair_pat<0, 3, 3>(v, f); break;
        case 0 | (4 << 3): pair_pat<0, 4, 3>(v, f); break;
        case 1 | (2 << 3): pair_pat<1, 2, 3>(v, f); break;
        case 1 | (3 << 3): pair_pat<1, 3, 3>(v, f); break;
        case 1 | (4 << 3): pair_pat<1, 4, 3>(v, f); break;
        case 2 | (3 << 3): pair_pat<2, 3, 3>(v, f); break;
        case 2 | (4 << 3): pair_pat<2, 4, 3>(v, f); break;
        default: pair_pat<3, 4, 3>(v, f); break;
    }
}

template <typename Off>
__device__ __forceinline__ bool op_applies(const TileOp &op, int tbits, Off base, unsigned condok) {
    if ((tbits & op.tmask) != op.tval) return false;
    if ((base & (Off)op.gmask) != (Off)op.gval) return false;
    if (op.cond != 0xffff && !((condok >> op.cond) & 1u)) return false;
    return true;
}

// global element offsets of the 32 registers: bits of r select strides
template <typename Off>
struct Offsets {
    Off o01[4], o23[4], s4;
    __device__ __forceinline__ void init(Off s0, Off s1, Off s2, Off s3, Off s4_) {
        o01[0] = 0; o01[1] = s0; o01[2] = s1; o01[3] = s0 + s1;
        o23[0] = 0; o23[1] = s2; o23[2] = s3; o23[3] = s2 + s3;
        s4 = s4_;
    }
    // register bit b of the index is inverted where bit b of f is set
    __device__ __forceinline__ void init_flipped(Off s0, Off s1, Off s2, Off s3, Off s4_, int f) {
        const Off a0 = (f & 1) ? s0 : 0, b0 = (f & 1) ? 0 : s0;   // offset of register bit 0 = 0 / 1
        const Off a1 = (f & 2) ? s1 : 0, b1 = (f & 2) ? 0 : s1;
        const Off a2 = (f & 4) ? s2 : 0, b2 = (f & 4) ? 0 : s2;
        const Off a3 = (f & 8) ? s3 : 0, b3 = (f & 8) ? 0 : s3;
        o01[0] = a0 + a1; o01[1] = b0 + a1; o01[2] = a0 + b1; o01[3] = b0 + b1;
        o23[0] = a2 + a3; o23[1] = b2 + a3; o23[2] = a2 + b3; o23[3] = b2 + b3;
        s4 = (f & 16) ? 0 : s4_;
        s4z = (f & 16) ? s4_ : 0;
    }
    Off s4z = 0;   // offset of register bit 4 = 0 (nonzero only when that bit is flipped)
    template <int r>
    __device__ __forceinline__ Off at() const {
        return o01[r & 3] + o23[(r >> 2) & 3] + ((r & 16) ? s4 : s4z);
    }
};

template <typename Off, int... rs>
__device__ __forceinline__ void load_all(const float2 *src, const Offsets<Off> &o, Regs &v,
                                         std::integer_sequence<int, rs...>) {
    float2 tmp[32];
    ((tmp[rs] = __ldcg(src + o.template at<rs>())), ...);
    ((re_of<rs>(v) = tmp[rs].x, im_of<rs>(v) = tmp[rs].y), ...);
}
template <typename Off, int... rs>
__device__ __forceinline__ void store_all(float2 *dst, const Offsets<Off> &o, Regs &v,
                                          std::integer_sequence<int, rs...>) {
    ((dst[o.template at<rs>()] = make_float2(re_of<rs>(v), im_of<rs>(v))), ...);
}

// Physical index of a tile's base (its local qubits 0): the tile index's bits
// deposited on the fixed qubits, one run of consecutive qubits at a time.
template <typename Head>
__device__ __forceinline__ uint64_t tile_base(const Head &P, uint64_t tile) {
    uint64_t b = 0;
#pragma unroll
    for (int r = 0; r < kTileMaxRuns; ++r)
        if (r < P.nruns) b |= ((tile >> P.run_tlo[r]) & ((1ull << P.run_len[r]) - 1)) << P.run_plo[r];
    return b;
}

// The op kinds a layered circuit rarely needs: controlled / conditioned 2x2
// gates, conditioned or complex pair factors, direct diagonal factors.
template <typename Off>
__device__ __forceinline__ void general_op(Regs &v, DevPending &pd, const TileOp &op, int tbits, Off base,
                                           unsigned condok) {
    if (op.kind == TOP_U2) {   // uniform part of the target's pending factor, in every thread
        pd.add(op.k, op.hturns);
        if (op.hmag != 1.f) bit_factor_dispatch(op.k, v, make_float2(op.hmag, 0.f));
    }
    if (!op_applies<Off>(op, tbits, base, condok)) return;
    if (op.kind == TOP_PAIR) {
        pair_dispatch(v, op.k, make_float2(op.ph.re, op.ph.im), op.rval);
        return;
    }
    if (op.kind == TOP_U2) {
        float2 m00 = make_float2(op.m[0], op.m[1]), m01 = make_float2(op.m[2], op.m[3]);
        float2 m10 = make_float2(op.m[4], op.m[5]), m11 = make_float2(op.m[6], op.m[7]);
        const int k = op.k;
        const uint32_t tk = pd.get(k);
        if (tk != 0u) {
            const float2 ak = phase_of(tk);
            if (op.rmask == 0) {  // fold diag(1, a_k) into the gate: U * diag(1, a_k)
                m01 = cmul(m01, ak);
                m11 = cmul(m11, ak);
            } else {
                bit_factor_dispatch(k, v, ak);
            }
        }
        pd.clear(k);
        if (k == 0) {
            u2_bit0(v, m00, m01, m10, m11, op.rmask, op.rval);
        } else {
            switch (k) {
                case 1: u2_packed<1>(v, m00, m01, m10, m11, op.rmask, op.rval); break;
                case 2: u2_packed<2>(v, m00, m01, m10, m11, op.rmask, op.rval); break;
                case 3: u2_packed<3>(v, m00, m01, m10, m11, op.rmask, op.rval); break;
                default: u2_packed<4>(v, m00, m01, m10, m11, op.rmask, op.rval); break;
            }
        }
    } else if (op.kind == TOP_PHASE) {  // factor where (register index & rmask) == rval
        const int rm = op.rmask;
        const int pc = __popc(rm);
        if (pc == 0) {
            pd.add(5, op.ph.turns);
        } else if (pc == 1) {
            const int k = __ffs(rm) - 1;
            if (op.rval) {
                pd.add(k, op.ph.turns);
            } else {  // f on bit k = 0:  f * (f^-1 on bit k = 1)
                pd.add(5, op.ph.turns);
                pd.add(k, 0u - op.ph.turns);
            }
        } else {
            const int rv = op.rval;
            const float2 f = make_float2(op.ph.re, op.ph.im);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                if (((2 * j) & rm) == rv) {
                    const float xr = v.R[j].x, xi = v.I[j].x;
                    v.R[j].x = xr * f.x - xi * f.y;
                    v.I[j].x = xr * f.y + xi * f.x;
                }
                if (((2 * j + 1) & rm) == rv) {
                    const float xr = v.R[j].y, xi = v.I[j].y;
                    v.R[j].y = xr * f.x - xi * f.y;
                    v.I[j].y = xr * f.y + xi * f.x;
                }
            }
        }
    }
}

// Where a pass program lives: in the kernel parameters (one state), or in
// device pools (a batched launch over many circuits).
struct ParamProg {
    const TileParams &P;
    __device__ __forceinline__ const TileHead &head() const { return P; }
    __device__ __forceinline__ const TileOp &op(int i) const { return P.ops[i]; }
    __device__ __forceinline__ const LayerGate &lg(int i) const { return P.lg[i]; }
    __device__ __forceinline__ const LinTerm &lin(int i) const { return P.lin[i]; }
};
struct PoolProg {
    const TileProg &h;
    const TileOp *ops;
    const LayerGate *lgs;
    const LinTerm *lins;
    __device__ __forceinline__ const TileProg &head() const { return h; }
    __device__ __forceinline__ const TileOp &op(int i) const { return ops[h.op0 + i]; }
    __device__ __forceinline__ const LayerGate &lg(int i) const { return lgs[h.lg0 + i]; }
    __device__ __forceinline__ const LinTerm &lin(int i) const { return lins[h.lin0 + i]; }
};

// The fields of a TileOp that the common op kinds read (its first 16 bytes),
// loaded as two 8-byte words.  The op loop loads the next op's head while the
// current op runs, so that a short op is not followed by a wait on the next
// op's fields.
struct OpHead {
    uint32_t w0, w1, w2, w3;
    __device__ __forceinline__ int kind() const { return (int)(w0 & 0xffu); }
    __device__ __forceinline__ int k() const { return (int)((w0 >> 8) & 0xffu); }
    __device__ __forceinline__ int rmask() const { return (int)((w0 >> 16) & 0xffu); }   // TOP_U2L: zf mask
    __device__ __forceinline__ int rval() const { return (int)(w0 >> 24); }
    __device__ __forceinline__ int count() const { return (int)(w2 >> 16); }
    __device__ __forceinline__ int first() const { return (int)(w3 & 0xffffu); }
    __device__ __forceinline__ int czmask() const { return (int)(w1 & 0x3ffu); }   // TOP_U2L: tmask
    __device__ __forceinline__ int count2() const { return (int)(w3 >> 16); }
};
__device__ __forceinline__ OpHead load_head(const TileOp &op) {
    const uint2 *p = reinterpret_cast<const uint2 *>(&op);
    const uint2 a = p[0], b = p[1];
    return OpHead{a.x, a.y, b.x, b.y};
}

// One tile of one pass: load, run the program, final flush, store.  GEN: the
// program may hold general ops (controlled or conditioned 2x2 gates, conditioned
// pair factors, direct diagonal factors); without them the kernel leaves their
// code out, which measured about 4 % faster on layer circuits (about 40 % less
// code in the op loop).
template <typename Off, bool GEN, typename Prog>
__device__ __forceinline__ void tile_body(const Prog &pr, float2 *__restrict__ psi, uint64_t tile,
                                          const uint8_t *__restrict__ cbits) {
    const auto &P = pr.head();
    // 2 x 2^13 floats (64 KiB) for transposes, then per thread six pending words
    extern __shared__ __align__(16) float smf[];
    float *sre = smf, *sim = smf + (1 << kTileQubits);
    uint32_t *spd = reinterpret_cast<uint32_t *>(smf + (2 << kTileQubits));     // pending sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tbits = (warp << 5) | lane;
    // lanes run over local qubits 0..4 in the load and store arrangements
    uint64_t lane_off = 0;
#pragma unroll
    for (int j = 0; j < 5; ++j)
        if ((lane >> j) & 1) lane_off += 1ull << P.S[j];

    {
        const Off base = (Off)tile_base(P, tile);

        // load in ARR_IO: lanes = local 0..4, registers = local 5..9, warps = local 10..12
        Regs v;
        {
            uint64_t tb = (uint64_t)base + lane_off;
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if ((warp >> j) & 1) tb += 1ull << P.S[10 + j];
            Offsets<Off> o;
            o.init((Off)1 << P.S[5], (Off)1 << P.S[6], (Off)1 << P.S[7], (Off)1 << P.S[8], (Off)1 << P.S[9]);
            load_all<Off>(psi + tb, o, v, std::make_integer_sequence<int, 32>{});
        }

        // while the loads are in flight: the phase table, the classical conditions
        if (P.need_tab) fill_turn_table();
        unsigned condok = 0;
        for (int c = 0; c < P.n_conds; ++c) {
            bool ok = true;
            for (int k = 0; k < P.conds[c].n; ++k) ok = ok && cbits[P.conds[c].idx[k]] != 0;
            condok |= (ok ? 1u : 0u) << c;
        }
        __syncthreads();

        DevPending pd;
        pd.p = spd + threadIdx.x;
        pd.reset();
        int cur = ARR_IO;
        const uint32_t tidx = (uint32_t)tile;
        OpHead nh{0u, 0u, 0u, 0u};
        if (P.nops > 0) nh = load_head(pr.op(0));
        for (int i = 0; i < P.nops; ++i) {
            const OpHead h = nh;
            if (i + 1 < P.nops) nh = load_head(pr.op(i + 1));
            switch (h.kind()) {
                case TOP_U2L: {
                    const LayerGate *lg = &pr.lg(h.first());
                    const int bits = h.k(), zf = h.rmask();
                    if (bits & 1) layer_gate<0>(v, pd, *lg++, zf & 1);
                    if (bits & 2) layer_gate<1>(v, pd, *lg++, zf & 2);
                    if (bits & 4) layer_gate<2>(v, pd, *lg++, zf & 4);
                    if (bits & 8) layer_gate<3>(v, pd, *lg++, zf & 8);
                    if (bits & 16) layer_gate<4>(v, pd, *lg, zf & 16);
                    if (h.czmask()) cz_mask(v, h.czmask());
                    break;
                }
                case TOP_PAIRNEG:
                    pair_neg(v, h.k());
                    break;
                case TOP_PHASEL: {
                    uint32_t acc = 0;
                    const int end = h.first() + h.count();
                    for (int e = h.first(); e < end; ++e) {
                        const LinTerm &L = pr.lin(e);
                        const bool ok = ((tbits & L.tmask) == L.tval) && ((tidx & L.fmask) == L.fval);
                        acc += ok ? L.turns : 0u;
                    }
                    if (acc) {
                        if (h.rval()) {  // the term's qubit is stored flipped: on bit k = 0
                            pd.add(5, acc);
                            pd.add(h.k(), 0u - acc);
                        } else {
                            pd.add(h.k(), acc);
                        }
                    }
                    break;
                }
                case TOP_PHASEB: {
                    const uint2 *t = reinterpret_cast<const uint2 *>(&pr.lin(0)) + h.first();
                    const int nt = h.count(), nf = h.count2();
                    uint32_t acc = 0, uacc = 0;
                    for (int e = 0; e < nt; ++e) {
                        const uint2 w = t[e];
                        acc += (((uint32_t)tbits >> w.x) & 1u) * w.y;
                    }
                    for (int e = nt; e < nt + nf; ++e) {
                        const uint2 w = t[e];
                        uacc += ((tidx >> w.x) & 1u) * w.y;
                    }
                    acc += uacc;
                    if (acc) {
                        if (h.rval()) {
                            pd.add(5, acc);
                            pd.add(h.k(), 0u - acc);
                        } else {
                            pd.add(h.k(), acc);
                        }
                    }
                    break;
                }
                case TOP_PAIRU: {
                    const float2 f = *reinterpret_cast<const float2 *>(&pr.op(i).ph.re);
                    pair11_dispatch(v, h.k(), f);
                    break;
                }
                case TOP_XPOSE:
                    flush_dev(v, pd);
                    transpose(v, sre, sim, cur, h.k(), lane, warp);
                    cur = h.k();
                    break;
                default:
                    if constexpr (GEN) general_op<Off>(v, pd, pr.op(i), tbits, base, condok);
                    break;
            }
        }

        // final flush: the thread's own pending phases plus the planner's uniform
        // factors (register bits, and lane / warp bits as a thread constant; each a
        // phase and a magnitude) and the pass's real scale.  The store arrangement is ARR_IO or ARR_HI: lanes =
        // local 0..4 in both; registers local 5..9 / 8..12, warps local 10..12 / 5..7.
        {
            const int rb = cur == ARR_IO ? 5 : 8, wb = cur == ARR_IO ? 10 : 5;
            uint32_t t0 = pd.get0() + P.fin_turns[13];
            float mg = P.fin_scale;   // the thread's constant magnitude
            for (uint64_t fm = P.fin_fixed_mask; fm; fm &= fm - 1) {
                const int b = __ffsll((long long)fm) - 1;
                if ((tile >> b) & 1) {
                    t0 += P.fin_fixed[b];
                    mg *= P.fin_fixed_mag[b];
                }
            }
#pragma unroll
            for (int j = 0; j < 5; ++j)
                if ((lane >> j) & 1) {
                    t0 += P.fin_turns[j];
                    mg *= P.fin_mag[j];
                }
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if ((warp >> j) & 1) {
                    t0 += P.fin_turns[wb + j];
                    mg *= P.fin_mag[wb + j];
                }
            float2 a[5];
            bool any = t0 != 0u || mg != 1.f;
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const uint32_t tk = pd.get(k) + P.fin_turns[rb + k];
                const float mk = P.fin_mag[rb + k];
                any = any || tk != 0u || mk != 1.f;
                const float2 e = phase_of(tk);
                a[k] = make_float2(e.x * mk, e.y * mk);
            }
            if (any) {
                const float2 c0 = phase_of(t0);
                apply_diagonal(v, make_float2(c0.x * mg, c0.y * mg), a);
            }
        }

        // store in ARR_IO or ARR_HI (lanes = local 0..4 in both); a local qubit the
        // planner left flipped has its index bit inverted here
        {
            const int fl = P.fin_flip;
            uint64_t tb = (uint64_t)base;
#pragma unroll
            for (int j = 0; j < 5; ++j)
                if (((lane ^ fl) >> j) & 1) tb += 1ull << P.S[j];
            const int rb = cur == ARR_IO ? 5 : 8, wb = cur == ARR_IO ? 10 : 5;
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (((warp ^ (fl >> wb)) >> j) & 1) tb += 1ull << P.S[wb + j];
            Offsets<Off> o;
            o.init_flipped((Off)1 << P.S[rb], (Off)1 << P.S[rb + 1], (Off)1 << P.S[rb + 2], (Off)1 << P.S[rb + 3],
                           (Off)1 << P.S[rb + 4], (fl >> rb) & 31);
            store_all<Off>(psi + tb, o, v, std::make_integer_sequence<int, 32>{});
        }
    }
}

// one tile per CTA (a grid-stride loop would keep the tile's addressing state
// live across iterations and push the kernel into spills)
template <typename Off, bool GEN>
__global__ void __launch_bounds__(kTileThreads, 2)
    k_tile(float2 *__restrict__ psi, const __grid_constant__ TileParams P, const uint8_t *__restrict__ cbits) {
    tile_body<Off, GEN>(ParamProg{P}, psi, blockIdx.x, cbits);
}

// Batched: CTA b finds its program by binary search in first[] (uniform over
// the CTA) and runs that program's tile b - first[c] on the program's state.
template <bool GEN>
__global__ void __launch_bounds__(kTileThreads, 2)
    k_tile_batch(const TileProg *__restrict__ progs, const uint32_t *__restrict__ first, int n_progs,
                 const TileOp *__restrict__ ops, const LayerGate *__restrict__ lg, const LinTerm *__restrict__ lin) {
    int lo = 0, hi = n_progs - 1;
    const uint32_t b = blockIdx.x;
    while (lo < hi) {  // the last c with first[c] <= b
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&first[mid]) <= b) lo = mid;
        else hi = mid - 1;
    }
    const TileProg &h = progs[lo];
    tile_body<uint32_t, GEN>(PoolProg{h, ops, lg, lin}, h.psi, b - __ldg(&first[lo]), nullptr);
}

// transposes (2^13 complex64) and pending sums (6 words per thread)
constexpr int kTileSmem = ((int)(2 * sizeof(float)) << kTileQubits) + 6 * kTileThreads * 4;

// the dynamic shared-memory attribute of kernel f, set once per device (host
// threads of the serving loop may launch concurrently; setting it twice is harmless)
template <typename F>
cudaError_t tile_smem_attr(F *f, std::atomic<bool> (&set)[64]) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!set[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmem);
        if (e != cudaSuccess) return e;
        set[dev].store(true, std::memory_order_release);
    }
    return cudaSuccess;
}

// whether a program needs the general-op path of the kernel
bool needs_general(const TileOp *ops, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (ops[i].kind == TOP_U2 || ops[i].kind == TOP_PHASE || ops[i].kind == TOP_PAIR) return true;
    return false;
}

template <typename Off, bool GEN>
cudaError_t launch_tile_g(void *psi, const TileParams &p, const uint8_t *cbits, cudaStream_t s) {
    static std::atomic<bool> attr_set[64];
    const cudaError_t e = tile_smem_attr(k_tile<Off, GEN>, attr_set);
    if (e != cudaSuccess) return e;
    k_tile<Off, GEN><<<(unsigned)p.n_tiles, kTileThreads, kTileSmem, s>>>((float2 *)psi, p, cbits);
    return cudaGetLastError();
}

template <typename Off>
cudaError_t launch_tile_t(void *psi, const TileParams &p, const uint8_t *cbits, cudaStream_t s) {
    if (p.n_tiles == 0 || p.n_tiles > (1ull << 31) - 1) return cudaErrorInvalidValue;
    if (p.nops < 0 || p.nops > kTileMaxOps) return cudaErrorInvalidValue;
    if (needs_general(p.ops, (size_t)p.nops)) return launch_tile_g<Off, true>(psi, p, cbits, s);
    return launch_tile_g<Off, false>(psi, p, cbits, s);
}

template <bool GEN>
cudaError_t launch_tile_batch_g(const TileProg *progs, const uint32_t *first, int n_progs, uint32_t n_ctas,
                                const TileOp *ops, const LayerGate *lg, const LinTerm *lin, cudaStream_t s) {
    static std::atomic<bool> attr_set[64];
    const cudaError_t e = tile_smem_attr(k_tile_batch<GEN>, attr_set);
    if (e != cudaSuccess) return e;
    k_tile_batch<GEN><<<n_ctas, kTileThreads, kTileSmem, s>>>(progs, first, n_progs, ops, lg, lin);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tile_batch(const TileProg *progs, const uint32_t *first, int n_progs, uint32_t n_ctas,
                              const TileOp *ops, const LayerGate *lg, const LinTerm *lin, bool general,
                              cudaStream_t s) {
    if (n_progs <= 0 || n_ctas == 0) return cudaSuccess;
    if (general) return launch_tile_batch_g<true>(progs, first, n_progs, n_ctas, ops, lg, lin, s);
    return launch_tile_batch_g<false>(progs, first, n_progs, n_ctas, ops, lg, lin, s);
}

bool tile_ops_need_general(const TileOp *ops, size_t n) { return needs_general(ops, n); }

cudaError_t launch_tile(void *psi, const TileParams &p, const uint8_t *cbits, cudaStream_t s) {
    // 32-bit element offsets inside a tile reach 2^32 amplitudes
    if (p.n <= 32) return launch_tile_t<uint32_t>(psi, p, cbits, s);
    return launch_tile_t<uint64_t>(psi, p, cbits, s);
}

}  // namespace qk
