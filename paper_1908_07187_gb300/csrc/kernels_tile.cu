// K3: fused tile pass for complex64 states.
//
// One CTA owns one tile of 2^13 amplitudes (13 physical qubits S[0..12], the
// other n-13 bits fixed by the tile index).  The tile is read from HBM once,
// a program of gates runs on it, and it is written back once, so a pass costs
// one read + one write of the state however many gates it carries.
//
// Amplitudes live in registers (32 per thread).  A 2x2 gate on a register bit
// is a butterfly between two registers of the same thread; the register bits
// are changed by transposing the tile through shared memory (three fixed
// arrangements, see qk_kernels.cuh).  Diagonal gates are not applied one by one:
// each thread keeps a factored diagonal -- a constant c0 and one factor a[k]
// per register bit -- and multiplies it into the amplitudes only when a
// non-commuting gate or a transpose needs it (a factor on the target bit of
// a 2x2 gate is folded into that gate's matrix instead).
#include <cuda_runtime.h>
#include <stdint.h>

#include "qk_kernels.cuh"

namespace qk {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cmac2(float2 m0, float2 a, float2 m1, float2 b) {
    float2 r;
    r.x = m0.x * a.x - m0.y * a.y + m1.x * b.x - m1.y * b.y;
    r.y = m0.x * a.y + m0.y * a.x + m1.x * b.y + m1.y * b.x;
    return r;
}

__host__ __device__ constexpr int ctz_const(int x) { return (x & 1) ? 0 : 1 + ctz_const(x >> 1); }

// Shared-memory slot of local index L: XOR-fold of the bits above 4 into the
// low 4 bits.  Every arrangement's warp access then touches 16 distinct 8-byte
// bank pairs per half warp (no conflicts).
__device__ __forceinline__ int swz(int L) { return L ^ (((L >> 4) ^ (L >> 8) ^ (L >> 12)) & 15); }

template <int ARR>
__device__ __forceinline__ int local_index(int r, int lane, int warp) {
    if constexpr (ARR == ARR_IO) return lane | (r << 5) | (warp << 10);
    else if constexpr (ARR == ARR_LO) return r | (lane << 5) | (warp << 10);
    else return lane | (r << 8) | (warp << 5);
}

template <int ARR>
__device__ __forceinline__ void to_smem(float2 *sm, const float2 (&v)[32], int lane, int warp) {
#pragma unroll
    for (int r = 0; r < 32; ++r) sm[swz(local_index<ARR>(r, lane, warp))] = v[r];
}

template <int ARR>
__device__ __forceinline__ void from_smem(const float2 *sm, float2 (&v)[32], int lane, int warp) {
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = sm[swz(local_index<ARR>(r, lane, warp))];
}

__device__ __forceinline__ void transpose(float2 (&v)[32], float2 *sm, int from, int to, int lane, int warp) {
    __syncthreads();
    if (from == ARR_IO) to_smem<ARR_IO>(sm, v, lane, warp);
    else if (from == ARR_LO) to_smem<ARR_LO>(sm, v, lane, warp);
    else to_smem<ARR_HI>(sm, v, lane, warp);
    __syncthreads();
    if (to == ARR_IO) from_smem<ARR_IO>(sm, v, lane, warp);
    else if (to == ARR_LO) from_smem<ARR_LO>(sm, v, lane, warp);
    else from_smem<ARR_HI>(sm, v, lane, warp);
}

// 2x2 butterfly on register bit K; with CTRL only for pairs whose register
// index has every bit of rmask set.
template <int K, bool CTRL>
__device__ __forceinline__ void u2_reg(float2 (&v)[32], float2 m00, float2 m01, float2 m10, float2 m11, int rmask) {
#pragma unroll
    for (int p = 0; p < 16; ++p) {
        const int r0 = ((p >> K) << (K + 1)) | (p & ((1 << K) - 1));
        const int r1 = r0 | (1 << K);
        if (!CTRL || (r0 & rmask) == rmask) {
            const float2 a = v[r0], b = v[r1];
            v[r0] = cmac2(m00, a, m01, b);
            v[r1] = cmac2(m10, a, m11, b);
        }
    }
}

template <bool CTRL>
__device__ __forceinline__ void u2_dispatch(int k, float2 (&v)[32], float2 m00, float2 m01, float2 m10, float2 m11,
                                            int rmask) {
    switch (k) {
        case 0: u2_reg<0, CTRL>(v, m00, m01, m10, m11, rmask); break;
        case 1: u2_reg<1, CTRL>(v, m00, m01, m10, m11, rmask); break;
        case 2: u2_reg<2, CTRL>(v, m00, m01, m10, m11, rmask); break;
        case 3: u2_reg<3, CTRL>(v, m00, m01, m10, m11, rmask); break;
        default: u2_reg<4, CTRL>(v, m00, m01, m10, m11, rmask); break;
    }
}

// v[r] *= f for every r with register bit K set
template <int K>
__device__ __forceinline__ void bit_factor(float2 (&v)[32], float2 f) {
#pragma unroll
    for (int r = 0; r < 32; ++r)
        if (r & (1 << K)) v[r] = cmul(v[r], f);
}

__device__ __forceinline__ void bit_factor_dispatch(int k, float2 (&v)[32], float2 f) {
    switch (k) {
        case 0: bit_factor<0>(v, f); break;
        case 1: bit_factor<1>(v, f); break;
        case 2: bit_factor<2>(v, f); break;
        case 3: bit_factor<3>(v, f); break;
        default: bit_factor<4>(v, f); break;
    }
}

// Pending factored diagonal of one thread: D(r) = c0 * prod_{k in r} a[k].
struct Pending {
    float2 c0;
    float2 a[5];
    int mask;  // bit k: a[k] != 1; bit 5: c0 != 1

    __device__ __forceinline__ void reset() {
        c0 = make_float2(1.f, 0.f);
#pragma unroll
        for (int k = 0; k < 5; ++k) a[k] = make_float2(1.f, 0.f);
        mask = 0;
    }
    __device__ __forceinline__ float2 get(int k) const {
        switch (k) {
            case 0: return a[0];
            case 1: return a[1];
            case 2: return a[2];
            case 3: return a[3];
            default: return a[4];
        }
    }
    __device__ __forceinline__ void mul(int k, float2 f) {
        switch (k) {
            case 0: a[0] = cmul(a[0], f); break;
            case 1: a[1] = cmul(a[1], f); break;
            case 2: a[2] = cmul(a[2], f); break;
            case 3: a[3] = cmul(a[3], f); break;
            default: a[4] = cmul(a[4], f); break;
        }
        mask |= 1 << k;
    }
    __device__ __forceinline__ void clear(int k) {
        switch (k) {
            case 0: a[0] = make_float2(1.f, 0.f); break;
            case 1: a[1] = make_float2(1.f, 0.f); break;
            case 2: a[2] = make_float2(1.f, 0.f); break;
            case 3: a[3] = make_float2(1.f, 0.f); break;
            default: a[4] = make_float2(1.f, 0.f); break;
        }
        mask &= ~(1 << k);
    }
    // multiply the whole pending diagonal into the registers
    __device__ __forceinline__ void flush(float2 (&v)[32]) {
        if (mask == 0) return;
        if ((mask & 32) == 0 && __popc(mask) <= 2) {
#pragma unroll
            for (int k = 0; k < 5; ++k)
                if (mask & (1 << k)) bit_factor_dispatch(k, v, a[k]);
        } else {
            // walk r in Gray-code order so that D(r) changes by one factor per step
            float2 d = c0;
            v[0] = cmul(v[0], d);
#pragma unroll
            for (int i = 1; i < 32; ++i) {
                const int g = i ^ (i >> 1), gp = (i - 1) ^ ((i - 1) >> 1);
                const int b = ctz_const(g ^ gp);
                d = cmul(d, (g & (1 << b)) ? a[b] : conjf2(a[b]));
                v[g] = cmul(v[g], d);
            }
        }
        reset();
    }
};

__device__ __forceinline__ bool op_applies(const TileOp &op, int tbits, uint64_t base, unsigned condok) {
    if ((tbits & op.tmask) != op.tval) return false;
    if ((base & op.gmask) != op.gval) return false;
    if (op.cond != 0xffff && !((condok >> op.cond) & 1u)) return false;
    return true;
}

__global__ void __launch_bounds__(kTileThreads, 2)
    k_tile(float2 *__restrict__ psi, const __grid_constant__ TileParams P, const uint8_t *__restrict__ cbits) {
    extern __shared__ __align__(16) float2 sm[];   // 2^13 amplitudes (64 KiB)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tbits = (warp << 5) | lane;

    unsigned condok = 0;
    for (int c = 0; c < P.n_conds; ++c) {
        bool ok = true;
        for (int k = 0; k < P.conds[c].n; ++k) ok = ok && cbits[P.conds[c].idx[k]] != 0;
        condok |= (ok ? 1u : 0u) << c;
    }

    for (uint64_t tile = blockIdx.x; tile < P.n_tiles; tile += gridDim.x) {
        uint64_t base = 0;
        for (int b = 0; b < P.nfix; ++b) base |= ((tile >> b) & 1ull) << P.fixed[b];

        // load in ARR_IO: lanes = local 0..4, registers = local 5..9, warps = local 10..12
        float2 v[32];
        {
            uint64_t tb = base + (uint64_t)lane;
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if ((warp >> j) & 1) tb += 1ull << P.S[10 + j];
            const float2 *src = psi + tb;
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                uint64_t off = 0;
#pragma unroll
                for (int k = 0; k < 5; ++k)
                    if ((r >> k) & 1) off += 1ull << P.S[5 + k];
                v[r] = src[off];
            }
        }

        Pending pd;
        pd.reset();
        int cur = ARR_IO;
        for (int i = 0; i < P.nops; ++i) {
            const TileOp &op = P.ops[i];
            if (op.kind == TOP_XPOSE) {
                pd.flush(v);
                transpose(v, sm, cur, op.k, lane, warp);
                cur = op.k;
                continue;
            }
            if (!op_applies(op, tbits, base, condok)) continue;
            if (op.kind == TOP_U2) {
                float2 m00 = make_float2(op.m[0], op.m[1]), m01 = make_float2(op.m[2], op.m[3]);
                float2 m10 = make_float2(op.m[4], op.m[5]), m11 = make_float2(op.m[6], op.m[7]);
                const int k = op.k;
                if (pd.mask & (1 << k)) {
                    const float2 ak = pd.get(k);
                    if (op.rmask == 0) {  // fold diag(1, a_k) into the gate: U * diag(1, a_k)
                        m01 = cmul(m01, ak);
                        m11 = cmul(m11, ak);
                    } else {
                        bit_factor_dispatch(k, v, ak);
                    }
                    pd.clear(k);
                }
                if (op.rmask) u2_dispatch<true>(k, v, m00, m01, m10, m11, op.rmask);
                else u2_dispatch<false>(k, v, m00, m01, m10, m11, 0);
            } else {  // TOP_PHASE: factor f where (register index & rmask) == rval
                const float2 f = make_float2(op.m[0], op.m[1]);
                const int rm = op.rmask;
                const int pc = __popc(rm);
                if (pc == 0) {
                    pd.c0 = cmul(pd.c0, f);
                    pd.mask |= 32;
                } else if (pc == 1) {
                    const int k = __ffs(rm) - 1;
                    if (op.rval) {
                        pd.mul(k, f);
                    } else {  // f on bit k = 0:  f * (f^-1 on bit k = 1)
                        pd.c0 = cmul(pd.c0, f);
                        pd.mask |= 32;
                        pd.mul(k, conjf2(f));
                    }
                } else {
                    const int rv = op.rval;
#pragma unroll
                    for (int r = 0; r < 32; ++r)
                        if ((r & rm) == rv) v[r] = cmul(v[r], f);
                }
            }
        }
        pd.flush(v);

        // store in ARR_IO or ARR_HI (lanes = local 0..4 in both)
        {
            uint64_t tb = base + (uint64_t)lane;
            if (cur == ARR_IO) {
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if ((warp >> j) & 1) tb += 1ull << P.S[10 + j];
                float2 *dst = psi + tb;
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    uint64_t off = 0;
#pragma unroll
                    for (int k = 0; k < 5; ++k)
                        if ((r >> k) & 1) off += 1ull << P.S[5 + k];
                    dst[off] = v[r];
                }
            } else {
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if ((warp >> j) & 1) tb += 1ull << P.S[5 + j];
                float2 *dst = psi + tb;
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    uint64_t off = 0;
#pragma unroll
                    for (int k = 0; k < 5; ++k)
                        if ((r >> k) & 1) off += 1ull << P.S[8 + k];
                    dst[off] = v[r];
                }
            }
        }
        __syncthreads();  // shared memory is reused by the next tile's transposes
    }
}

}  // namespace

cudaError_t launch_tile(void *psi, const TileParams &p, const uint8_t *cbits, cudaStream_t s) {
    constexpr int smem = (int)sizeof(float2) << kTileQubits;
    static bool attr_set = false;  // per process; the attribute is per function
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    uint64_t grid = p.n_tiles;
    if (grid > (1ull << 30)) grid = 1ull << 30;
    k_tile<<<(unsigned)grid, kTileThreads, smem, s>>>((float2 *)psi, p, cbits);
    return cudaGetLastError();
}

}  // namespace qk
