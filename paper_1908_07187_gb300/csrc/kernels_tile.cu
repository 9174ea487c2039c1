// K3: fused tile pass for complex64 states.
//
// One CTA owns one tile of 2^13 amplitudes (13 physical qubits S[0..12]; the
// other n-13 bits are fixed by the tile index).  The tile is read from HBM once,
// a program of gates runs on it, and it is written back once, so a pass costs
// one read + one write of the state however many gates it carries.
//
// Each of the 256 threads holds 32 amplitudes in registers, split into real and
// imaginary parts, two amplitudes per float2 (re[2j], re[2j+1]) /
// (im[2j], im[2j+1]).  A 2x2 gate on a register bit is a set of 16 butterflies
// between registers of the same thread (scalar FP32 FMAs: the paired f32x2 forms
// measured slower in this register-bound loop).  The register bits are changed
// by transposing the tile through shared memory (three fixed arrangements, see
// qk_kernels.cuh).
//
// Diagonal gates are not applied one by one: each thread keeps a pending
// diagonal D(r) = exp(2 pi i (t0 + sum_{k in r} t_k) / 2^32) as six 32-bit
// fixed-point phase sums (exact modulo one turn), and multiplies it into the
// amplitudes only when a transpose or a gate that does not commute with it needs
// that; a pending factor on the target bit of a 2x2 gate is folded into the
// gate's matrix instead.
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "qk_kernels.cuh"

namespace qk {
namespace {

__host__ __device__ constexpr int ctz_const(int x) { return (x & 1) ? 0 : 1 + ctz_const(x >> 1); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 splat(float x) { return make_float2(x, x); }

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

struct Mat {
    float2 a00r, a00i, n00i, a01r, a01i, n01i, a10r, a10i, n10i, a11r, a11i, n11i;
    __device__ __forceinline__ Mat(float2 m00, float2 m01, float2 m10, float2 m11) {
        a00r = splat(m00.x); a00i = splat(m00.y); n00i = splat(-m00.y);
        a01r = splat(m01.x); a01i = splat(m01.y); n01i = splat(-m01.y);
        a10r = splat(m10.x); a10i = splat(m10.y); n10i = splat(-m10.y);
        a11r = splat(m11.x); a11i = splat(m11.y); n11i = splat(-m11.y);
    }
};

// 2x2 gate on register bit K >= 1: couples (j, j | 2^(K-1)) of float2 registers,
// two amplitude pairs per couple.  A couple acts if (2j & rmask) == rmask;
// with register bit 0 in rmask only the odd halves act (the even halves keep
// their old values).
template <int K>
__device__ __forceinline__ void u2_packed(Regs &v, const Mat &M, int rmask) {
    static_assert(K >= 1 && K <= 4, "packed butterflies need K >= 1");
    const bool odd_only = rmask & 1;
    const int hmask = rmask & ~1;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (j & (1 << (K - 1))) continue;
        const int j1 = j | (1 << (K - 1));
        if (((j << 1) & hmask) != hmask) continue;
        const float2 A = v.R[j], B = v.I[j], C = v.R[j1], D = v.I[j1];
        // scalar FMAs measured faster than the paired forms here
        float2 r0, i0, r1, i1;
        r0.x = M.a00r.x * A.x + M.n00i.x * B.x + M.a01r.x * C.x + M.n01i.x * D.x;
        r0.y = M.a00r.x * A.y + M.n00i.x * B.y + M.a01r.x * C.y + M.n01i.x * D.y;
        i0.x = M.a00r.x * B.x + M.a00i.x * A.x + M.a01r.x * D.x + M.a01i.x * C.x;
        i0.y = M.a00r.x * B.y + M.a00i.x * A.y + M.a01r.x * D.y + M.a01i.x * C.y;
        r1.x = M.a10r.x * A.x + M.n10i.x * B.x + M.a11r.x * C.x + M.n11i.x * D.x;
        r1.y = M.a10r.x * A.y + M.n10i.x * B.y + M.a11r.x * C.y + M.n11i.x * D.y;
        i1.x = M.a10r.x * B.x + M.a10i.x * A.x + M.a11r.x * D.x + M.a11i.x * C.x;
        i1.y = M.a10r.x * B.y + M.a10i.x * A.y + M.a11r.x * D.y + M.a11i.x * C.y;
        if (odd_only) {
            r0.x = A.x; i0.x = B.x; r1.x = C.x; i1.x = D.x;
        }
        v.R[j] = r0; v.I[j] = i0; v.R[j1] = r1; v.I[j1] = i1;
    }
}

// 2x2 gate on register bit 0: the pair is the two halves of one packed register.
__device__ __forceinline__ void u2_bit0(Regs &v, float2 m00, float2 m01, float2 m10, float2 m11, int rmask) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (((j << 1) & rmask) != rmask) continue;
        const float2 a = make_float2(v.R[j].x, v.I[j].x), b = make_float2(v.R[j].y, v.I[j].y);
        const float2 o0 = make_float2(m00.x * a.x - m00.y * a.y + m01.x * b.x - m01.y * b.y,
                                      m00.x * a.y + m00.y * a.x + m01.x * b.y + m01.y * b.x);
        const float2 o1 = make_float2(m10.x * a.x - m10.y * a.y + m11.x * b.x - m11.y * b.y,
                                      m10.x * a.y + m10.y * a.x + m11.x * b.y + m11.y * b.x);
        v.R[j] = make_float2(o0.x, o1.x);
        v.I[j] = make_float2(o0.y, o1.y);
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
            v.R[j] = __ffma2_rn(nfi, B, __fmul2_rn(fr, A));
            v.I[j] = __ffma2_rn(fi, A, __fmul2_rn(fr, B));
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

// Pending diagonal of one thread in 32-bit fixed-point turns.  The six sums live
// in shared memory (word w of thread x at w * kTileThreads + x, conflict-free),
// leaving the registers to the amplitudes; only the mask is a register.
struct Pending {
    uint32_t *p;  // word 0: t0 (constant), word 1 + k: t_k (register bit k)
    float2 *fa;   // flush scratch: factor k at fa[k * kTileThreads]
    int mask;     // bit k: t_k may be nonzero; bit 5: t0 may be nonzero

    __device__ __forceinline__ uint32_t &t0() { return p[0]; }
    __device__ __forceinline__ uint32_t &t(int k) { return p[(k + 1) * kTileThreads]; }
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int w = 0; w < 6; ++w) p[w * kTileThreads] = 0;
        mask = 0;
    }
    __device__ __forceinline__ void add(int k, uint32_t d) {
        t(k) += d;
        mask |= 1 << k;
    }
    __device__ __forceinline__ void add0(uint32_t d) {
        t0() += d;
        mask |= 32;
    }
    __device__ __forceinline__ void clear(int k) {
        t(k) = 0;
        mask &= ~(1 << k);
    }
    __device__ __forceinline__ void flush(Regs &v) {
        if (mask == 0) return;
        if ((mask & 32) == 0 && __popc(mask) <= 2) {
#pragma unroll
            for (int k = 0; k < 5; ++k)
                if (mask & (1 << k)) {
                    const uint32_t tk = t(k);
                    if (tk != 0) bit_factor_dispatch(k, v, turns_to_phase(tk));
                }
        } else {
            // D(r) = c0 * prod_{k in r} a_k: six sincos into this thread's factor
            // slots in shared memory (not registers: the amplitudes fill those), then
            // walk j (register bits 1..4) in Gray-code order so D changes by one factor
            // per step
            const float2 c0 = (mask & 32) ? turns_to_phase(t0()) : make_float2(1.f, 0.f);
#pragma unroll
            for (int k = 0; k < 5; ++k)
                fa[k * kTileThreads] = (mask & (1 << k)) ? turns_to_phase(t(k)) : make_float2(1.f, 0.f);
            const float2 a0 = fa[0];
            // four independent chains over register bits 1, 2 (j = 4h + l, l < 4),
            // started at c0 * (a3, a4 products of h): dependency depth 4, not 16
            float2 d[4];
            {
                const float2 a3 = fa[3 * kTileThreads], a4 = fa[4 * kTileThreads];
                d[0] = c0;
                d[1] = cmul(c0, a3);
                d[2] = cmul(c0, a4);
                d[3] = cmul(d[1], a4);
            }
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                // l walks 0, 1, 3, 2 (Gray order over bits 1 and 2)
                const int g = l ^ (l >> 1);
                if (l > 0) {
                    const int gp = (l - 1) ^ ((l - 1) >> 1);
                    const int bb = ctz_const(g ^ gp);      // register bit bb + 1 toggles
                    const float2 ab = fa[(bb + 1) * kTileThreads];
                    const float2 f = (g >> bb) & 1 ? ab : make_float2(ab.x, -ab.y);
#pragma unroll
                    for (int h = 0; h < 4; ++h) d[h] = cmul(d[h], f);
                }
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int j = 4 * h + g;
                    const float2 d1 = cmul(d[h], a0);
                    const float2 Dr = make_float2(d[h].x, d1.x), Di = make_float2(d[h].y, d1.y);
                    const float2 A = v.R[j], B = v.I[j];
                    v.R[j] = __ffma2_rn(make_float2(-Di.x, -Di.y), B, __fmul2_rn(Dr, A));
                    v.I[j] = __ffma2_rn(Di, A, __fmul2_rn(Dr, B));
                }
            }
        }
        reset();
    }
};

// Rotation butterfly on register bit K: (x0, x1) <- (c x0 + m01 x1, s x0 + m11 x1)
// with c, s real and m01, m11 complex: 12 FP32 operations per amplitude pair.
template <int K>
__device__ __forceinline__ void rot_butterfly(Regs &v, float c, float s, float2 m01, float2 m11) {
    const float n01i = -m01.y, n11i = -m11.y;
    if constexpr (K == 0) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float ar = v.R[j].x, ai = v.I[j].x, br = v.R[j].y, bi = v.I[j].y;
            v.R[j].x = fmaf(n01i, bi, fmaf(m01.x, br, c * ar));
            v.I[j].x = fmaf(m01.y, br, fmaf(m01.x, bi, c * ai));
            v.R[j].y = fmaf(n11i, bi, fmaf(m11.x, br, s * ar));
            v.I[j].y = fmaf(m11.y, br, fmaf(m11.x, bi, s * ai));
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j & (1 << (K - 1))) continue;
            const int j1 = j | (1 << (K - 1));
            const float2 A = v.R[j], B = v.I[j], C = v.R[j1], D = v.I[j1];
            float2 r0, i0, r1, i1;
            r0.x = fmaf(n01i, D.x, fmaf(m01.x, C.x, c * A.x));
            r0.y = fmaf(n01i, D.y, fmaf(m01.x, C.y, c * A.y));
            i0.x = fmaf(m01.y, C.x, fmaf(m01.x, D.x, c * B.x));
            i0.y = fmaf(m01.y, C.y, fmaf(m01.x, D.y, c * B.y));
            r1.x = fmaf(n11i, D.x, fmaf(m11.x, C.x, s * A.x));
            r1.y = fmaf(n11i, D.y, fmaf(m11.x, C.y, s * A.y));
            i1.x = fmaf(m11.y, C.x, fmaf(m11.x, D.x, s * B.x));
            i1.y = fmaf(m11.y, C.y, fmaf(m11.x, D.y, s * B.y));
            v.R[j] = r0; v.I[j] = i0; v.R[j1] = r1; v.I[j1] = i1;
        }
    }
}

// One gate of a TOP_U2L layer on register bit K, given in rotation form
// U = e^{i a} diag(1, e^{i p}) [[c, -s], [s, c]] diag(1, e^{i l}) (m = c, s, then a, p,
// l as 32-bit turns).  The right factor and the pending phase of bit K fold into the
// butterfly, U diag(1, b) with b = e^{i l} times the pending factor; the left
// factors become the new pending phases of bit K and of the whole thread (folded
// into the next gate on that bit, or flushed at the next transpose).  A variant
// that applied the left factor inside the butterfly when no later gate on the bit
// follows measured slower: the second code path raised register spills.
template <int K>
__device__ __forceinline__ void layer_gate(Regs &v, Pending &pd, const float *m) {
    const float c = m[0], s = m[1];
    const uint32_t ta = __float_as_uint(m[2]), tp = __float_as_uint(m[3]);
    uint32_t tb = __float_as_uint(m[4]);
    if (pd.mask & (1 << K)) tb += pd.t(K);
    float2 m01 = make_float2(-s, 0.f), m11 = make_float2(c, 0.f);
    if (tb != 0) {
        const float2 b = turns_to_phase(tb);
        m01 = make_float2(-s * b.x, -s * b.y);
        m11 = make_float2(c * b.x, c * b.y);
    }
    rot_butterfly<K>(v, c, s, m01, m11);
    pd.t(K) = tp;
    if (tp != 0) pd.mask |= 1 << K;
    else pd.mask &= ~(1 << K);
    if (ta != 0) pd.add0(ta);
}

// amplitudes whose register bits K and L are both 1 are multiplied by f (or negated)
template <int K, int L, int r>
__device__ __forceinline__ void pair_one(Regs &v, float2 f, bool neg) {
    if constexpr (((r >> K) & 1) && ((r >> L) & 1)) {
        float &x = re_of<r>(v);
        float &y = im_of<r>(v);
        if (neg) {
            x = -x;
            y = -y;
        } else {
            const float xr = x, xi = y;
            x = xr * f.x - xi * f.y;
            y = xr * f.y + xi * f.x;
        }
    }
}
template <int K, int L, int... rs>
__device__ __forceinline__ void pair_all(Regs &v, float2 f, bool neg, std::integer_sequence<int, rs...>) {
    (pair_one<K, L, rs>(v, f, neg), ...);
}
template <int K, int L>
__device__ __forceinline__ void pair_factor(Regs &v, float2 f, bool neg) {
    pair_all<K, L>(v, f, neg, std::make_integer_sequence<int, 32>{});
}

// fixed-bit masks and the tile base in the offset width (32 bits while n <= 32)
template <typename Off>
__device__ __forceinline__ Off ld_mask(const uint64_t *p) {
    if constexpr (sizeof(Off) == 4) return __ldg(reinterpret_cast<const uint32_t *>(p));  // low word
    else return __ldg(reinterpret_cast<const unsigned long long *>(p));
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
    template <int r>
    __device__ __forceinline__ Off at() const {
        return o01[r & 3] + o23[(r >> 2) & 3] + ((r & 16) ? s4 : (Off)0);
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

template <typename Off>
__global__ void __launch_bounds__(kTileThreads, 2)
    k_tile(float2 *__restrict__ psi, const __grid_constant__ TileParams P, const TileEntries *__restrict__ tab,
           const uint8_t *__restrict__ cbits) {
    // 2 x 2^13 floats (64 KiB) for transposes, then per thread five flush factors, six
    // pending words and one word per TOP_PHASES op
    extern __shared__ __align__(16) float smf[];
    float *sre = smf, *sim = smf + (1 << kTileQubits);
    float2 *sfa = reinterpret_cast<float2 *>(smf + (2 << kTileQubits));       // flush factors
    uint32_t *spd = reinterpret_cast<uint32_t *>(sfa + 5 * kTileThreads);       // pending sums
    uint32_t *sph = spd + 6 * kTileThreads;                                      // phase-op sums
    uint32_t *spat = sph + P.nphops * kTileThreads;                              // pattern sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tbits = (warp << 5) | lane;
    // lanes run over local qubits 0..4 in the load and store arrangements
    uint64_t lane_off = 0;
#pragma unroll
    for (int j = 0; j < 5; ++j)
        if ((lane >> j) & 1) lane_off += 1ull << P.S[j];

    fill_turn_table();
    __syncthreads();

    unsigned condok = 0;
    for (int c = 0; c < P.n_conds; ++c) {
        bool ok = true;
        for (int k = 0; k < P.conds[c].n; ++k) ok = ok && cbits[P.conds[c].idx[k]] != 0;
        condok |= (ok ? 1u : 0u) << c;
    }

    for (uint64_t tile = blockIdx.x; tile < P.n_tiles; tile += gridDim.x) {
        uint64_t base64 = 0;
        for (int b = 0; b < P.nfix; ++b) base64 |= ((tile >> b) & 1ull) << P.fixed[b];
        const Off base = (Off)base64;

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

        // the pass's phase sums for this tile and thread, while the loads are in flight:
        // one thread per pattern adds its fixed-bit-conditioned terms (uniform over the
        // tile), then every thread adds the patterns whose thread-bit condition it meets
        if (P.nphops) {
            for (int q = threadIdx.x; q < P.npats; q += kTileThreads) {
                const PhasePattern pt = tab->p[q];
                uint32_t sum = pt.turns;
                const int ende = pt.first + pt.count;
                for (int e = pt.first; e < ende; ++e) {
                    const Off gm = ld_mask<Off>(&tab->e[e].gmask), gv = ld_mask<Off>(&tab->e[e].gval);
                    const uint32_t tu = __ldg(&tab->e[e].turns);
                    sum += ((base & gm) == gv) ? tu : 0u;
                }
                spat[q] = sum;
            }
            __syncthreads();
            for (int slot = 0; slot < P.nphops; ++slot) {
                uint32_t acc = 0;
                const int endp = P.phop[slot][0] + P.phop[slot][1];
                for (int q = P.phop[slot][0]; q < endp; ++q) {
                    const PhasePattern &pt = P.pats[q];
                    acc += ((tbits & pt.tmask) == pt.tval) ? spat[q] : 0u;
                }
                sph[slot * kTileThreads + threadIdx.x] = acc;
            }
        }

        Pending pd;
        pd.p = spd + threadIdx.x;
        pd.fa = sfa + threadIdx.x;
        pd.reset();
        int cur = ARR_IO;
        for (int i = 0; i < P.nops; ++i) {
            const TileOp &op = P.ops[i];
            if (op.kind == TOP_XPOSE) {
                pd.flush(v);
                transpose(v, sre, sim, cur, op.k, lane, warp);
                cur = op.k;
                continue;
            }
            if (op.kind == TOP_U2L) {
                const float *mp = P.mats[op.first];
                const int bits = op.k;
                if (bits & 1) { layer_gate<0>(v, pd, mp); mp += 8; }
                if (bits & 2) { layer_gate<1>(v, pd, mp); mp += 8; }
                if (bits & 4) { layer_gate<2>(v, pd, mp); mp += 8; }
                if (bits & 8) { layer_gate<3>(v, pd, mp); mp += 8; }
                if (bits & 16) layer_gate<4>(v, pd, mp);
                continue;
            }
            if (op.kind == TOP_PHASES) {
                const uint32_t acc = sph[op.count2 * kTileThreads + threadIdx.x];
                if (op.k == 5) {
                    pd.add0(acc);
                } else {
                    pd.add(op.k, acc);
                }
                continue;
            }
            if (!op_applies<Off>(op, tbits, base, condok)) continue;
            if (op.kind == TOP_PAIR) {
                const float2 f = make_float2(op.ph.re, op.ph.im);
                const bool neg = op.ph.turns == 0x80000000u;
                switch (op.k) {
                    case 0 | (1 << 3): pair_factor<0, 1>(v, f, neg); break;
                    case 0 | (2 << 3): pair_factor<0, 2>(v, f, neg); break;
                    case 0 | (3 << 3): pair_factor<0, 3>(v, f, neg); break;
                    case 0 | (4 << 3): pair_factor<0, 4>(v, f, neg); break;
                    case 1 | (2 << 3): pair_factor<1, 2>(v, f, neg); break;
                    case 1 | (3 << 3): pair_factor<1, 3>(v, f, neg); break;
                    case 1 | (4 << 3): pair_factor<1, 4>(v, f, neg); break;
                    case 2 | (3 << 3): pair_factor<2, 3>(v, f, neg); break;
                    case 2 | (4 << 3): pair_factor<2, 4>(v, f, neg); break;
                    default: pair_factor<3, 4>(v, f, neg); break;
                }
                continue;
            }
            if (op.kind == TOP_U2) {
                float2 m00 = make_float2(op.m[0], op.m[1]), m01 = make_float2(op.m[2], op.m[3]);
                float2 m10 = make_float2(op.m[4], op.m[5]), m11 = make_float2(op.m[6], op.m[7]);
                const int k = op.k;
                if (pd.mask & (1 << k)) {
                    const uint32_t tk = pd.t(k);
                    if (tk != 0) {
                        const float2 ak = turns_to_phase(tk);
                        if (op.rmask == 0) {  // fold diag(1, a_k) into the gate: U * diag(1, a_k)
                            m01 = cmul(m01, ak);
                            m11 = cmul(m11, ak);
                        } else {
                            bit_factor_dispatch(k, v, ak);
                        }
                    }
                    pd.clear(k);
                }
                if (k == 0) {
                    u2_bit0(v, m00, m01, m10, m11, op.rmask);
                } else {
                    const Mat M(m00, m01, m10, m11);
                    switch (k) {
                        case 1: u2_packed<1>(v, M, op.rmask); break;
                        case 2: u2_packed<2>(v, M, op.rmask); break;
                        case 3: u2_packed<3>(v, M, op.rmask); break;
                        default: u2_packed<4>(v, M, op.rmask); break;
                    }
                }
            } else if (op.kind == TOP_PHASE) {  // factor where (register index & rmask) == rval
                const int rm = op.rmask;
                const int pc = __popc(rm);
                if (pc == 0) {
                    pd.add0(op.ph.turns);
                } else if (pc == 1) {
                    const int k = __ffs(rm) - 1;
                    if (op.rval) {
                        pd.add(k, op.ph.turns);
                    } else {  // f on bit k = 0:  f * (f^-1 on bit k = 1)
                        pd.add0(op.ph.turns);
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
        pd.flush(v);

        // store in ARR_IO or ARR_HI (lanes = local 0..4 in both)
        {
            uint64_t tb = (uint64_t)base + lane_off;
            Offsets<Off> o;
            if (cur == ARR_IO) {
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if ((warp >> j) & 1) tb += 1ull << P.S[10 + j];
                o.init((Off)1 << P.S[5], (Off)1 << P.S[6], (Off)1 << P.S[7], (Off)1 << P.S[8], (Off)1 << P.S[9]);
            } else {
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if ((warp >> j) & 1) tb += 1ull << P.S[5 + j];
                o.init((Off)1 << P.S[8], (Off)1 << P.S[9], (Off)1 << P.S[10], (Off)1 << P.S[11], (Off)1 << P.S[12]);
            }
            store_all<Off>(psi + tb, o, v, std::make_integer_sequence<int, 32>{});
        }
        __syncthreads();  // shared memory is reused by the next tile's transposes
    }
}

__global__ void k_tile_entries(const __grid_constant__ TileEntries E, int ne, int np, TileEntries *__restrict__ dst) {
    for (int i = threadIdx.x; i < ne; i += blockDim.x) dst->e[i] = E.e[i];
    for (int i = threadIdx.x; i < np; i += blockDim.x) dst->p[i] = E.p[i];
}

template <typename Off>
cudaError_t launch_tile_t(void *psi, const TileParams &p, const TileEntries *entries, const uint8_t *cbits,
                          cudaStream_t s) {
    // transposes (2^13 complex64), flush factors (5 float2), pending (6 words), phase sums
    constexpr int smem_max =
        ((int)(2 * sizeof(float)) << kTileQubits) + (16 + kTileMaxPhOps) * kTileThreads * 4 + kTileMaxPats * 4;
    const int smem = ((int)(2 * sizeof(float)) << kTileQubits) + (16 + p.nphops) * kTileThreads * 4 +
                     (p.nphops ? p.npats * 4 : 0);
    // the shared-memory attribute is set once per device
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        e = cudaFuncSetAttribute(k_tile<Off>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    uint64_t grid = p.n_tiles;
    if (grid > (1ull << 30)) grid = 1ull << 30;
    k_tile<Off><<<(unsigned)grid, kTileThreads, smem, s>>>((float2 *)psi, p, entries, cbits);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tile(void *psi, const TileParams &p, const TileEntries *entries, const uint8_t *cbits,
                        cudaStream_t s) {
    // 32-bit element offsets inside a tile reach 2^32 amplitudes
    if (p.n <= 32) return launch_tile_t<uint32_t>(psi, p, entries, cbits, s);
    return launch_tile_t<uint64_t>(psi, p, entries, cbits, s);
}

cudaError_t launch_tile_entries(const TileEntries &e, int nentries, int npats, TileEntries *dst, cudaStream_t s) {
    if (nentries <= 0 && npats <= 0) return cudaSuccess;
    k_tile_entries<<<1, 256, 0, s>>>(e, nentries, npats, dst);
    return cudaGetLastError();
}

}  // namespace qk
