// One-pass-per-gate kernels of libqk: 2x2 pair updates (K1), diagonal phases
// (K2), dense k-qubit blocks, permutation gathers (K5), measurement (K6), and
// small helpers.  Every kernel streams the amplitudes it touches once, with
// 16-byte vector accesses where the qubit layout allows.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "qk_kernels.cuh"

namespace qk {
namespace {

constexpr int kThreads = 256;

template <typename R> struct Amp;
template <> struct Amp<float> { using T = float2; };
template <> struct Amp<double> { using T = double2; };

template <typename T>
__device__ __forceinline__ T cmul(T a, T b) {
    T r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// out = m0 * a + m1 * b
template <typename T>
__device__ __forceinline__ T cmac2(T m0, T a, T m1, T b) {
    T r;
    r.x = m0.x * a.x - m0.y * a.y + m1.x * b.x - m1.y * b.y;
    r.y = m0.x * a.y + m0.y * a.x + m1.x * b.y + m1.y * b.x;
    return r;
}

__device__ __forceinline__ bool cond_ok(const Cond &c, const uint8_t *cbits) {
    for (int k = 0; k < c.n; ++k)
        if (cbits[c.idx[k]] == 0) return false;
    return true;
}

// Insert a zero bit at each sorted position (ascending) of p into j.
__device__ __forceinline__ uint64_t insert_zeros(uint64_t j, const Positions &p) {
    for (int k = 0; k < p.n; ++k) {
        const uint64_t lo = j & ((1ull << p.pos[k]) - 1);
        j = ((j - lo) << 1) | lo;
    }
    return j;
}

inline unsigned grid_for(uint64_t units, int sms, int per_sm = 16) {
    uint64_t b = (units + kThreads - 1) / kThreads;
    uint64_t cap = (uint64_t)sms * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// ---------------------------------------------------------------------------
// K1: 2x2 update on pairs (i0, i0 + 2^q) where every control bit is 1.
// V = 0: generic, one pair per unit, scalar amplitude accesses.
// V = 1: complex64, q == 0: the pair is one 16-byte vector.
// V = 2: complex64, q >= 1 and bit 0 free: two adjacent pairs per unit, two
//        16-byte vectors.
// ---------------------------------------------------------------------------
template <typename R, int V>
__global__ void __launch_bounds__(kThreads) k_u2(typename Amp<R>::T *psi, U2Args a, const uint8_t *cbits) {
    using T = typename Amp<R>::T;
    if (a.cond.n && !cond_ok(a.cond, cbits)) return;
    T m00, m01, m10, m11;
    m00.x = (R)a.m[0]; m00.y = (R)a.m[1];
    m01.x = (R)a.m[2]; m01.y = (R)a.m[3];
    m10.x = (R)a.m[4]; m10.y = (R)a.m[5];
    m11.x = (R)a.m[6]; m11.y = (R)a.m[7];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t qbit = 1ull << a.q;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < a.n_units; u += stride) {
        if constexpr (V == 1) {
            const uint64_t i0 = insert_zeros(u, a.ins) | a.cmask;
            float4 *p = reinterpret_cast<float4 *>(psi + i0);
            float4 v = *p;
            T x0 = make_float2(v.x, v.y), x1 = make_float2(v.z, v.w);
            T y0 = cmac2(m00, x0, m01, x1), y1 = cmac2(m10, x0, m11, x1);
            *p = make_float4(y0.x, y0.y, y1.x, y1.y);
        } else if constexpr (V == 2) {
            const uint64_t i0 = insert_zeros(u << 1, a.ins) | a.cmask;
            float4 *p0 = reinterpret_cast<float4 *>(psi + i0);
            float4 *p1 = reinterpret_cast<float4 *>(psi + (i0 | qbit));
            float4 v0 = *p0, v1 = *p1;
            T a0 = make_float2(v0.x, v0.y), b0 = make_float2(v1.x, v1.y);
            T a1 = make_float2(v0.z, v0.w), b1 = make_float2(v1.z, v1.w);
            T ya0 = cmac2(m00, a0, m01, b0), yb0 = cmac2(m10, a0, m11, b0);
            T ya1 = cmac2(m00, a1, m01, b1), yb1 = cmac2(m10, a1, m11, b1);
            *p0 = make_float4(ya0.x, ya0.y, ya1.x, ya1.y);
            *p1 = make_float4(yb0.x, yb0.y, yb1.x, yb1.y);
        } else {
            const uint64_t i0 = insert_zeros(u, a.ins) | a.cmask;
            const uint64_t i1 = i0 | qbit;
            T x0 = psi[i0], x1 = psi[i1];
            psi[i0] = cmac2(m00, x0, m01, x1);
            psi[i1] = cmac2(m10, x0, m11, x1);
        }
    }
}

// ---------------------------------------------------------------------------
// K2: multiply amplitudes with (i & mask) == val by a phase factor.
// V = 0 generic (one amplitude per unit); V = 1 complex64 with bit 0 outside
// the mask (two adjacent amplitudes per unit, one 16-byte vector).
// With n_rphase > 0 the factor is exp(-2 pi i sum_l c_l / 2^(l+1)) from cbits.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ typename Amp<R>::T phase_factor(const PhaseArgs &a, const uint8_t *cbits) {
    typename Amp<R>::T f;
    if (a.n_rphase == 0) {
        f.x = (R)a.f_re;
        f.y = (R)a.f_im;
        return f;
    }
    // fraction of a turn in 64-bit fixed point: sum_l c_l 2^-(l+1), l = 1..e
    uint64_t turns = 0;
    for (int l = 1; l <= a.n_rphase; ++l)
        if (cbits[a.rphase_idx[l - 1]]) turns += 1ull << (63 - l);
    const double frac = (double)turns * 0x1p-64;  // in [0, 1/2)
    double s, c;
    sincospi(-2.0 * frac, &s, &c);
    f.x = (R)c;
    f.y = (R)s;
    return f;
}

template <typename R, int V>
__global__ void __launch_bounds__(kThreads) k_phase(typename Amp<R>::T *psi, PhaseArgs a, const uint8_t *cbits) {
    using T = typename Amp<R>::T;
    if (a.cond.n && !cond_ok(a.cond, cbits)) return;
    // an angle from cbits is formed in FP64 once per block (GB300's FP64 rate is low)
    __shared__ T s_f;
    if (a.n_rphase) {
        if (threadIdx.x == 0) s_f = phase_factor<R>(a, cbits);
        __syncthreads();
    }
    const T f = a.n_rphase ? s_f : phase_factor<R>(a, cbits);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < a.n_units; u += stride) {
        if constexpr (V == 1) {
            const uint64_t i = insert_zeros(u << 1, a.ins) | a.val;
            float4 *p = reinterpret_cast<float4 *>(psi + i);
            float4 v = *p;
            T x0 = cmul(make_float2(v.x, v.y), f), x1 = cmul(make_float2(v.z, v.w), f);
            *p = make_float4(x0.x, x0.y, x1.x, x1.y);
        } else {
            const uint64_t i = insert_zeros(u, a.ins) | a.val;
            psi[i] = cmul(psi[i], f);
        }
    }
}

// ---------------------------------------------------------------------------
// Dense k-qubit block.  Each block iteration handles 256 / 2^k groups with one
// thread per output amplitude: the group vectors are staged in shared memory,
// thread (g, r) forms row r of M v_g.  The matrix sits in shared memory too.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kThreads) k_matk(typename Amp<R>::T *psi, MatKArgs a, const uint8_t *cbits) {
    using T = typename Amp<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K = a.k, G = 1 << K;
    T *mat = reinterpret_cast<T *>(smem_raw);
    T *vec = mat + G * G;
    if (a.cond.n && !cond_ok(a.cond, cbits)) return;
    const T *gm = reinterpret_cast<const T *>(a.mat);
    for (int e = threadIdx.x; e < G * G; e += blockDim.x) mat[e] = gm[e];
    const int gpb = kThreads >> K;          // groups per block iteration
    const int g = threadIdx.x >> K, r = threadIdx.x & (G - 1);
    uint64_t off = 0;                       // offset of register value r
    for (int b = 0; b < K; ++b)
        if ((r >> (K - 1 - b)) & 1) off |= 1ull << a.tpos[b];
    for (uint64_t g0 = (uint64_t)blockIdx.x * gpb; g0 < a.n_groups; g0 += (uint64_t)gridDim.x * gpb) {
        const uint64_t grp = g0 + g;
        const bool live = grp < a.n_groups;
        const uint64_t idx = live ? ((insert_zeros(grp, a.ins) | a.cmask) | off) : 0;
        __syncthreads();
        if (live) vec[threadIdx.x] = psi[idx];
        __syncthreads();
        if (live) {
            T acc;
            acc.x = 0;
            acc.y = 0;
            const T *row = mat + r * G;
            const T *v = vec + g * G;
            for (int c = 0; c < G; ++c) {
                const T m = row[c], x = v[c];
                acc.x += m.x * x.x - m.y * x.y;
                acc.y += m.x * x.y + m.y * x.x;
            }
            psi[idx] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// K5: controlled register permutation as an out-of-place gather:
// out[i] = in[src(i)], src replacing the register value y by f^-1(y).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mulmod_barrett(uint64_t x, uint64_t y, uint64_t N, uint64_t mu) {
    const uint64_t p = x * y;                  // x, y < 2^30: exact
    const uint64_t q = __umul64hi(p, mu);      // floor(p / N) - {0, 1, 2}
    uint64_t r = p - q * N;
    while (r >= N) r -= N;
    return r;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_perm(const typename Amp<R>::T *__restrict__ in,
                                                   typename Amp<R>::T *__restrict__ out, PermArgs a,
                                                   const uint8_t *cbits) {
    const bool active = (a.cond.n == 0) || cond_ok(a.cond, cbits);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_amps; i += stride) {
        uint64_t src = i;
        if (active && (i & a.cmask) == a.cmask) {
            uint64_t y = 0;
            if (a.field.contig) {
                y = field_get(i, a.field, a.w);
            } else {
                for (int b = 0; b < a.w; ++b) y = (y << 1) | ((i >> a.rpos[b]) & 1u);
            }
            uint64_t x = y;
            if (a.kind == 0) {
                if (y < a.N) x = mulmod_barrett(a.cinv, y, a.N, a.mu);
            } else {
                x = a.finv[y];
            }
            if (a.field.contig) {
                src = field_put(src, x, a.field, a.w);
            } else {
                for (int b = 0; b < a.w; ++b) {
                    const uint64_t bit = (x >> (a.w - 1 - b)) & 1u;
                    src = (src & ~(1ull << a.rpos[b])) | (bit << a.rpos[b]);
                }
            }
        }
        out[i] = in[src];
    }
}

// Modular exponentiation (ModExpArgs): one out-of-place gather for a whole run of
// controlled multiplications on one register.  The group tables go to shared
// memory once per block (their indices differ from lane to lane).
template <typename R>
__global__ void __launch_bounds__(kThreads) k_modexp(const typename Amp<R>::T *__restrict__ in,
                                                     typename Amp<R>::T *__restrict__ out,
                                                     const __grid_constant__ ModExpArgs a, const uint8_t *cbits) {
    __shared__ uint32_t tab[kModExpGroups * 256];
    for (int k = threadIdx.x; k < a.ngroups * 256; k += blockDim.x) tab[k] = a.tab[k >> 8][k & 255];
    __syncthreads();
    const bool active = (a.cond.n == 0) || cond_ok(a.cond, cbits);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_amps; i += stride) {
        uint64_t src = i;
        if (active) {
            uint64_t y = 0;
            if (a.field.contig) {
                y = field_get(i, a.field, a.w);
            } else {
                for (int b = 0; b < a.w; ++b) y = (y << 1) | ((i >> a.rpos[b]) & 1u);
            }
            if (y < a.N) {
                uint64_t m = 1;
                for (int g = 0; g < a.ngroups; ++g) {
                    uint32_t v = 0;
                    const int j0 = 8 * g, j1 = min(a.nctl, j0 + 8);
                    for (int j = j0; j < j1; ++j) v |= (uint32_t)((i >> a.cpos[j]) & 1u) << (j - j0);
                    const uint64_t t = tab[(g << 8) | v];
                    m = g == 0 ? t : mulmod_barrett(m, t, a.N, a.mu);
                }
                const uint64_t x = mulmod_barrett(m, y, a.N, a.mu);
                if (a.field.contig) {
                    src = field_put(src, x, a.field, a.w);
                } else {
                    for (int b = 0; b < a.w; ++b) {
                        const uint64_t bit = (x >> (a.w - 1 - b)) & 1u;
                        src = (src & ~(1ull << a.rpos[b])) | (bit << a.rpos[b]);
                    }
                }
            }
        }
        out[i] = in[src];
    }
}

// ---------------------------------------------------------------------------
// K6: measurement.  reduce -> per-block (S0, S1); the last block to finish adds
// the block partials in a fixed order (so results do not depend on timing) and
// decides; collapse.  complex64 sums run in compensated FP32 (a float pair that
// carries each addition's rounding error, about twice float's precision) and
// reach FP64 once per thread: GB300 has 2 FP64 lanes per SM per clock.
// ---------------------------------------------------------------------------
// prefix value of the decided outcomes: sum_j m_j << pos[j], j < k
__device__ __forceinline__ uint64_t prefix_value(const MeasArgs &a, const MeasSlot *slots, int k) {
    uint64_t v = 0;
    for (int j = 0; j < k; ++j) v |= (uint64_t)(slots[j].m & 1) << a.pos[j];
    return v;
}

__device__ __forceinline__ uint64_t insert_bits(uint64_t j, const MeasArgs &a) {
    for (int t = 0; t < a.nins; ++t) {
        const uint64_t lo = j & ((1ull << a.ins[t]) - 1);
        j = ((j - lo) << 1) | lo;
    }
    return j;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_meas_reduce(const typename Amp<R>::T *__restrict__ psi, MeasArgs a,
                                                          const MeasSlot *slots, double *partials, Decide dec) {
    __shared__ double sh[kThreads];
    const uint64_t pv = prefix_value(a, slots, a.k);
    const int q = a.pos[a.k];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool bit0_free = a.nins == 0 || a.ins[0] != 0;
    double d0 = 0.0, d1 = 0.0;
    if constexpr (sizeof(R) == 4) {
        // complex64: |a|^2 in FP32, compensated FP32 running sums (FP64 only per thread)
        FSum g0, g1;
        if (bit0_free && a.n_units >= 2) {
            // two adjacent amplitudes (one 16-byte vector) per unit
            const uint64_t n_units = a.n_units >> 1;
#pragma unroll 4
            for (uint64_t u = tid; u < n_units; u += stride) {
                const uint64_t i = insert_bits(u << 1, a) | pv;
                const float4 v = *reinterpret_cast<const float4 *>(psi + i);
                const float pa = v.x * v.x + v.y * v.y, pb = v.z * v.z + v.w * v.w;
                if (q == 0) {
                    g0.add(pa);
                    g1.add(pb);
                } else if ((i >> q) & 1u) {
                    g1.add(pa + pb);
                } else {
                    g0.add(pa + pb);
                }
            }
        } else {
            for (uint64_t u = tid; u < a.n_units; u += stride) {
                const uint64_t i = insert_bits(u, a) | pv;
                const typename Amp<R>::T v = psi[i];
                const float pa = v.x * v.x + v.y * v.y;
                if ((i >> q) & 1u) g1.add(pa); else g0.add(pa);
            }
        }
        d0 = g0.value();
        d1 = g1.value();
    } else {
        for (uint64_t u = tid; u < a.n_units; u += stride) {
            const uint64_t i = insert_bits(u, a) | pv;
            const typename Amp<R>::T v = psi[i];
            const double pa = (double)v.x * v.x + (double)v.y * v.y;
            if ((i >> q) & 1u) d1 += pa; else d0 += pa;
        }
    }
    const double s0 = block_sum_w0(d0, sh);
    const double s1 = block_sum_w0(d1, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = s0;
        partials[2 * blockIdx.x + 1] = s1;
    }
    last_block_decides(partials, dec);
}

// Project onto the decided outcomes of every measured qubit and renormalise:
// amplitudes that match keep a * 1/sqrt(P), the others are written as zero
// without being read.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_meas_collapse(typename Amp<R>::T *psi, uint64_t n_amps, MeasArgs a,
                                                            const MeasSlot *slots) {
    uint64_t M = 0;
    for (int j = 0; j < a.k; ++j) M |= 1ull << a.pos[j];
    const uint64_t V = prefix_value(a, slots, a.k);
    const R sc = (R)slots[a.k - 1].scale;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (sizeof(R) == 4) {
        float4 *p = reinterpret_cast<float4 *>(psi);
        for (uint64_t u = tid; u < (n_amps >> 1); u += stride) {
            const uint64_t i = u << 1;
            const bool ka = (i & M) == V, kb = ((i + 1) & M) == V;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ka || kb) {
                v = p[u];
                const float sa = ka ? sc : 0.f, sb = kb ? sc : 0.f;
                v.x *= sa; v.y *= sa; v.z *= sb; v.w *= sb;
            }
            p[u] = v;
        }
    } else {
        for (uint64_t i = tid; i < n_amps; i += stride) {
            typename Amp<R>::T v;
            v.x = 0;
            v.y = 0;
            if ((i & M) == V) {
                v = psi[i];
                v.x *= sc;
                v.y *= sc;
            }
            psi[i] = v;
        }
    }
}

template <typename R>
__global__ void k_set_basis(typename Amp<R>::T *psi, uint64_t index) {
    typename Amp<R>::T one;
    one.x = 1;
    one.y = 0;
    psi[index] = one;
}

// The same permutation, tiled: a tile is every value of the output bits that
// are the five lowest or come from the five lowest input bits (m <= 10 bits),
// the other bits fixed.  Its 2^m amplitudes are read as runs along the input low
// bits and written as runs along the output low bits, through shared memory.
struct RelabelTiled {
    int m, n_other;
    uint64_t n_tiles;
    int other_out[40], other_in[40];   // tile-index bit t -> output bit / input bit
    uint64_t in_off[1024];             // input offset of tile element u (input-local order)
    uint64_t out_off[1024];            // output offset of tile element v (output-local order)
    uint16_t src_of[1024];             // input-local index of output-local element v
};

// Tiled relabel (RelabelTiled): persistent CTAs, offset tables in shared memory;
// the tile buffer is XOR-swizzled on its low five index bits so that reads along
// either side's runs stay conflict-free.
__device__ __forceinline__ int relabel_slot(int u) { return u ^ ((u >> 5) & 31); }

template <typename R>
__global__ void __launch_bounds__(kThreads) k_relabel_tiled(const typename Amp<R>::T *__restrict__ in,
                                                            typename Amp<R>::T *__restrict__ out,
                                                            const __grid_constant__ RelabelTiled a) {
    using T = typename Amp<R>::T;
    __shared__ uint64_t s_in[1024], s_out[1024];
    __shared__ uint16_t s_src[1024];
    __shared__ T buf[1024];
    const int M = 1 << a.m;
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        s_in[k] = a.in_off[k];
        s_out[k] = a.out_off[k];
        s_src[k] = a.src_of[k];
    }
    __syncthreads();
    for (uint64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        uint64_t bin = 0, bout = 0;
        for (int t = 0; t < a.n_other; ++t)
            if ((tile >> t) & 1u) {
                bin |= 1ull << a.other_in[t];
                bout |= 1ull << a.other_out[t];
            }
        for (int u = threadIdx.x; u < M; u += blockDim.x) buf[relabel_slot(u)] = in[bin + s_in[u]];
        __syncthreads();
        for (int v = threadIdx.x; v < M; v += blockDim.x) out[bout + s_out[v]] = buf[relabel_slot(s_src[v])];
        __syncthreads();
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_u2(int prec, void *psi, const U2Args &a, const uint8_t *cbits, int n, int sms,
                      cudaStream_t s) {
    (void)n;
    if (prec == 0) {
        const bool bit0_control = (a.cmask & 1ull) != 0;
        if (a.q == 0) {
            k_u2<float, 1><<<grid_for(a.n_units, sms), kThreads, 0, s>>>((float2 *)psi, a, cbits);
        } else if (!bit0_control && a.n_units >= 2) {
            U2Args b = a;
            b.n_units = a.n_units >> 1;
            k_u2<float, 2><<<grid_for(b.n_units, sms), kThreads, 0, s>>>((float2 *)psi, b, cbits);
        } else {
            k_u2<float, 0><<<grid_for(a.n_units, sms), kThreads, 0, s>>>((float2 *)psi, a, cbits);
        }
    } else {
        k_u2<double, 0><<<grid_for(a.n_units, sms), kThreads, 0, s>>>((double2 *)psi, a, cbits);
    }
    return cudaGetLastError();
}

cudaError_t launch_phase(int prec, void *psi, const PhaseArgs &a, const uint8_t *cbits, int sms,
                         cudaStream_t s) {
    if (prec == 0) {
        if ((a.mask & 1ull) == 0 && a.n_units >= 2) {
            PhaseArgs b = a;
            b.n_units = a.n_units >> 1;
            k_phase<float, 1><<<grid_for(b.n_units, sms), kThreads, 0, s>>>((float2 *)psi, b, cbits);
        } else {
            k_phase<float, 0><<<grid_for(a.n_units, sms), kThreads, 0, s>>>((float2 *)psi, a, cbits);
        }
    } else {
        k_phase<double, 0><<<grid_for(a.n_units, sms), kThreads, 0, s>>>((double2 *)psi, a, cbits);
    }
    return cudaGetLastError();
}

template <typename R>
static cudaError_t matk_r(void *psi, const MatKArgs &a, const uint8_t *cbits, int sms, cudaStream_t s) {
    using T = typename Amp<R>::T;
    if (a.k < 1 || a.k > 6) return cudaErrorInvalidValue;
    const size_t sm = sizeof(T) * (((size_t)1 << (2 * a.k)) + kThreads);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_matk<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    const uint64_t gpb = kThreads >> a.k;
    uint64_t blocks = (a.n_groups + gpb - 1) / gpb;
    if (blocks > (uint64_t)sms * 8) blocks = (uint64_t)sms * 8;
    k_matk<R><<<(unsigned)blocks, kThreads, sm, s>>>((T *)psi, a, cbits);
    return cudaGetLastError();
}

cudaError_t launch_matk(int prec, void *psi, const MatKArgs &a, const uint8_t *cbits, int sms,
                        cudaStream_t s) {
    return prec == 0 ? matk_r<float>(psi, a, cbits, sms, s) : matk_r<double>(psi, a, cbits, sms, s);
}

cudaError_t launch_modexp(int prec, const void *in, void *out, const ModExpArgs &a, const uint8_t *cbits, int sms,
                          cudaStream_t s) {
    if (prec == 0)
        k_modexp<float><<<grid_for(a.n_amps, sms), kThreads, 0, s>>>((const float2 *)in, (float2 *)out, a, cbits);
    else
        k_modexp<double><<<grid_for(a.n_amps, sms), kThreads, 0, s>>>((const double2 *)in, (double2 *)out, a, cbits);
    return cudaGetLastError();
}

cudaError_t launch_perm(int prec, const void *in, void *out, const PermArgs &a, const uint8_t *cbits,
                        int sms, cudaStream_t s) {
    if (prec == 0)
        k_perm<float><<<grid_for(a.n_amps, sms), kThreads, 0, s>>>((const float2 *)in, (float2 *)out, a, cbits);
    else
        k_perm<double><<<grid_for(a.n_amps, sms), kThreads, 0, s>>>((const double2 *)in, (double2 *)out, a, cbits);
    return cudaGetLastError();
}

cudaError_t launch_measure_reduce(int prec, const void *psi, int n, const MeasArgs &a, const MeasSlot *slots,
                                  double *partials, int nblocks, const Decide &d, cudaStream_t s) {
    if (n < 1) return cudaErrorInvalidValue;
    if (prec == 0)
        k_meas_reduce<float><<<nblocks, kThreads, 0, s>>>((const float2 *)psi, a, slots, partials, d);
    else
        k_meas_reduce<double><<<nblocks, kThreads, 0, s>>>((const double2 *)psi, a, slots, partials, d);
    return cudaGetLastError();
}

cudaError_t launch_measure_collapse(int prec, void *psi, int n, const MeasArgs &a, const MeasSlot *slots, int sms,
                                    cudaStream_t s) {
    const uint64_t n_amps = 1ull << n;
    if (prec == 0)
        k_meas_collapse<float><<<grid_for(n_amps >> 1, sms), kThreads, 0, s>>>((float2 *)psi, n_amps, a, slots);
    else
        k_meas_collapse<double><<<grid_for(n_amps, sms), kThreads, 0, s>>>((double2 *)psi, n_amps, a, slots);
    return cudaGetLastError();
}

cudaError_t launch_set_basis(int prec, void *psi, uint64_t index, cudaStream_t s) {
    if (prec == 0)
        k_set_basis<float><<<1, 1, 0, s>>>((float2 *)psi, index);
    else
        k_set_basis<double><<<1, 1, 0, s>>>((double2 *)psi, index);
    return cudaGetLastError();
}

cudaError_t launch_relabel(int prec, const void *in, void *out, const RelabelArgs &a, int sms,
                           cudaStream_t s) {
    // tile bits: output bits 0..4 and the output bits fed by input bits 0..4
    const int n = a.n, lo = n < 5 ? n : 5;
    int inv[64];
    for (int j = 0; j < n; ++j) inv[a.phys_of[j]] = j;   // input bit -> output bit
    bool in_tile[64] = {false};
    int out_bits[10], m = 0;
    for (int j = 0; j < lo; ++j) { in_tile[j] = true; out_bits[m++] = j; }
    for (int i = 0; i < lo; ++i)
        if (!in_tile[inv[i]]) { in_tile[inv[i]] = true; out_bits[m++] = inv[i]; }
    int in_bits[10], mi = 0;
    bool in_used[64] = {false};
    for (int i = 0; i < lo; ++i) { in_used[i] = true; in_bits[mi++] = i; }
    for (int k = 0; k < m; ++k) {
        const int i = a.phys_of[out_bits[k]];
        if (!in_used[i]) { in_used[i] = true; in_bits[mi++] = i; }
    }
    if (mi != m) return cudaErrorInvalidValue;        // cannot happen for a permutation
    static thread_local RelabelTiled t;
    t.m = m;
    t.n_other = 0;
    for (int j = 0; j < n; ++j)
        if (!in_tile[j]) {
            t.other_out[t.n_other] = j;
            t.other_in[t.n_other] = a.phys_of[j];
            ++t.n_other;
        }
    t.n_tiles = 1ull << t.n_other;
    int in_pos[64];                                    // input bit -> input-local position
    for (int k = 0; k < m; ++k) in_pos[in_bits[k]] = k;
    for (int u = 0; u < (1 << m); ++u) {
        uint64_t off = 0;
        for (int k = 0; k < m; ++k)
            if ((u >> k) & 1) off |= 1ull << in_bits[k];
        t.in_off[u] = off;
    }
    for (int v = 0; v < (1 << m); ++v) {
        uint64_t off = 0;
        int u = 0;
        for (int k = 0; k < m; ++k)
            if ((v >> k) & 1) {
                off |= 1ull << out_bits[k];
                u |= 1 << in_pos[a.phys_of[out_bits[k]]];
            }
        t.out_off[v] = off;
        t.src_of[v] = (uint16_t)u;
    }
    // each CTA copies the offset tables once: give it at least about 8 tiles
    // (small states), at most 8 CTAs per SM (large ones)
    uint64_t want = (uint64_t)sms * 8;
    const uint64_t per8 = t.n_tiles / 8 > (uint64_t)sms ? t.n_tiles / 8 : (uint64_t)sms;
    if (per8 < want) want = per8;
    const unsigned grid = (unsigned)(t.n_tiles < want ? t.n_tiles : want);
    if (prec == 0)
        k_relabel_tiled<float><<<grid, kThreads, 0, s>>>((const float2 *)in, (float2 *)out, t);
    else
        k_relabel_tiled<double><<<grid, kThreads, 0, s>>>((const double2 *)in, (double2 *)out, t);
    return cudaGetLastError();
}

}  // namespace qk
