// K7: one fused stage of Kitaev's one-control-qubit order finding.
//
// The generic stage is H(c); controlled x -> f(x) on the register; the
// semiclassical phase exp(i theta) on c = |1>; H(c); measure c; X(c) if the
// outcome is 1.  When c is |0> at the start (it is reset at the end of every
// stage), with w the amplitudes on c = 0 and v = U w (v(y) = w(f^-1(y))), the
// state just before the measurement is
//     c = 0:  (w + e^{i theta} v) / 2,     c = 1:  (w - e^{i theta} v) / 2,
// so one reduction gives s0 = sum |w + e^{i theta} v|^2 and s1 = sum |w - ...|^2,
// P0 = s0 / (s0 + s1), and after the outcome m and the reset the c = 0 amplitudes
// are (w + (-1)^m e^{i theta} v) / sqrt(s_m).  Two passes over the c = 0 half
// replace six gate passes.
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

__device__ __forceinline__ uint64_t insert_zero(uint64_t j, int pos) {
    const uint64_t lo = j & ((1ull << pos) - 1);
    return ((j - lo) << 1) | lo;
}

__device__ __forceinline__ uint64_t mulmod_barrett(uint64_t x, uint64_t y, uint64_t N, uint64_t mu) {
    const uint64_t p = x * y;                  // x, y < 2^30: exact
    const uint64_t q = __umul64hi(p, mu);      // floor(p / N) - {0, 1, 2}
    uint64_t r = p - q * N;
    while (r >= N) r -= N;
    return r;
}

// index of the amplitude whose register value is f^-1(register value of i)
__device__ __forceinline__ uint64_t source_index(uint64_t i, const KitaevArgs &a) {
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
    if (a.field.contig) return field_put(i, x, a.field, a.w);
    uint64_t src = i;
    for (int b = 0; b < a.w; ++b) {
        const uint64_t bit = (x >> (a.w - 1 - b)) & 1u;
        src = (src & ~(1ull << a.rpos[b])) | (bit << a.rpos[b]);
    }
    return src;
}

// exp(i theta), theta = -2 pi sum_l c_l / 2^(l+1) from the listed cbits (64-bit fixed point)
__device__ __forceinline__ double2 rphase(const KitaevArgs &a, const uint8_t *cbits) {
    uint64_t turns = 0;
    for (int l = 1; l <= a.n_rphase; ++l)
        if (cbits[a.rphase_idx[l - 1]]) turns += 1ull << (63 - l);
    double s, c;
    sincospi(-2.0 * ((double)turns * 0x1p-64), &s, &c);
    return make_double2(c, s);
}

// the stage's phase factor, formed in FP64 by one thread per block (GB300's FP64
// rate is low) and shared
__device__ __forceinline__ double2 block_rphase(const KitaevArgs &a, const uint8_t *cbits) {
    __shared__ double2 s_om;
    if (threadIdx.x == 0) s_om = rphase(a, cbits);
    __syncthreads();
    return s_om;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_kitaev_reduce(const typename Amp<R>::T *__restrict__ psi, KitaevArgs a,
                                                            const uint8_t *cbits, double *partials, Decide dec) {
    __shared__ double sh[kThreads];
    const double2 om = block_rphase(a, cbits);
    const R wr = (R)om.x, wi = (R)om.y;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // complex64: compensated FP32 sums; complex128: FP64
    FSum g0, g1;
    double d0 = 0.0, d1 = 0.0;
#pragma unroll 4
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.n_half; j += stride) {
        const uint64_t i = insert_zero(j, a.cpos);   // control bit 0
        const typename Amp<R>::T w = psi[i], v = psi[source_index(i, a)];
        const R tr = wr * v.x - wi * v.y, ti = wr * v.y + wi * v.x;
        const R pr = w.x + tr, pi = w.y + ti, mr = w.x - tr, mi = w.y - ti;
        if constexpr (sizeof(R) == 4) {
            g0.add(pr * pr + pi * pi);
            g1.add(mr * mr + mi * mi);
        } else {
            d0 += pr * pr + pi * pi;
            d1 += mr * mr + mi * mi;
        }
    }
    if constexpr (sizeof(R) == 4) {
        d0 = g0.value();
        d1 = g1.value();
    }
    const double s0 = block_sum_w0(d0, sh);
    const double s1 = block_sum_w0(d1, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = s0;
        partials[2 * blockIdx.x + 1] = s1;
    }
    last_block_decides(partials, dec);
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_kitaev_update(const typename Amp<R>::T *__restrict__ psi,
                                                            typename Amp<R>::T *__restrict__ out, KitaevArgs a,
                                                            const uint8_t *cbits, const MeasSlot *slot) {
    // the decision and the phase, converted to the working precision once per block
    __shared__ R s_f[3];
    {
        const double2 om = block_rphase(a, cbits);
        if (threadIdx.x == 0) {
            const double sg = slot->m ? -1.0 : 1.0;
            s_f[0] = (R)slot->scale;
            s_f[1] = (R)(sg * om.x);
            s_f[2] = (R)(sg * om.y);
        }
        __syncthreads();
    }
    const R sc = s_f[0], wr = s_f[1], wi = s_f[2];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.n_half; j += stride) {
        const uint64_t i = insert_zero(j, a.cpos);
        const typename Amp<R>::T w = psi[i], v = psi[source_index(i, a)];
        typename Amp<R>::T o, z;
        o.x = (w.x + wr * v.x - wi * v.y) * sc;
        o.y = (w.y + wr * v.y + wi * v.x) * sc;
        z.x = 0;
        z.y = 0;
        out[i] = o;                         // control back at |0>
        out[i | (1ull << a.cpos)] = z;
    }
}

inline unsigned grid_for(uint64_t units, int sms) {
    uint64_t b = (units + kThreads - 1) / kThreads;
    const uint64_t cap = (uint64_t)sms * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

cudaError_t launch_kitaev_reduce(int prec, const void *psi, const KitaevArgs &a, const uint8_t *cbits,
                                 double *partials, int nblocks, const Decide &d, cudaStream_t s) {
    if (prec == 0)
        k_kitaev_reduce<float><<<nblocks, kThreads, 0, s>>>((const float2 *)psi, a, cbits, partials, d);
    else
        k_kitaev_reduce<double><<<nblocks, kThreads, 0, s>>>((const double2 *)psi, a, cbits, partials, d);
    return cudaGetLastError();
}

cudaError_t launch_kitaev_update(int prec, const void *psi, void *out, const KitaevArgs &a, const uint8_t *cbits,
                                 const MeasSlot *slot, int sms, cudaStream_t s) {
    if (prec == 0)
        k_kitaev_update<float><<<grid_for(a.n_half, sms), kThreads, 0, s>>>((const float2 *)psi, (float2 *)out, a,
                                                                            cbits, slot);
    else
        k_kitaev_update<double><<<grid_for(a.n_half, sms), kThreads, 0, s>>>((const double2 *)psi, (double2 *)out,
                                                                             a, cbits, slot);
    return cudaGetLastError();
}

}  // namespace qk
