// K4, tensor-core form: a dense 5-qubit complex64 unitary U on the five lowest
// physical qubits, applied as a batched complex matrix product on tcgen05.
//
// The state is a matrix of 2^(n-5) group rows; a row holds the 32 amplitudes
// that share the upper bits, stored as 64 interleaved floats (re, im).  With the
// real 64 x 64 embedding B of U (B[2x][2r] = Re U[r][x], B[2x+1][2r] = -Im U,
// B[2x][2r+1] = Im U, B[2x+1][2r+1] = Re U) every row becomes Y = X B, i.e. a
// GEMM with M = 2^(n-5), N = K = 64.  TF32 tensor cores keep 10 mantissa bits,
// so the product uses the 3xTF32 split X = Xh + Xl, B = Bh + Bl (Xh, Bh the
// inputs with the low 13 mantissa bits cleared) and D = Xh Bh + Xh Bl + Xl Bh in
// FP32, close to full FP32 accuracy (Markidis et al., "NVIDIA Tensor Core
// programmability, performance & precision", 2018).
//
// One persistent CTA per SM, its warps specialised and pipelined: 128-row tiles
// of X arrive by TMA (128-byte swizzle) into a three-stage shared-memory ring;
// four warps write Xl beside each; one thread issues 24 tcgen05.mma (3 products
// x 8 K-steps of 8) into one of two 128 x 64 FP32 accumulators in tensor memory;
// four other warps read a finished accumulator back with tcgen05.ld and store it
// in place while the next tile's products run.  Every mbarrier wait has an
// iteration limit; on timeout the kernel records an error, waits (bounded) for
// its own copies in flight, releases its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "qk_kernels.cuh"

namespace qk {
namespace {

constexpr int kRows = 128;                    // rows per tile = MMA M
constexpr int kCols = 64;                     // floats per row = MMA K = MMA N
constexpr int kChunk = kRows * 128;           // one 128-byte-wide K chunk of the tile (16 KiB)
constexpr int kTile = 2 * kChunk;             // 32 KiB
constexpr int kBChunk = kCols * 128;          // 8 KiB
constexpr int kB = 2 * kBChunk;               // 16 KiB
constexpr int kThreads = 320;                 // 10 warps: producer, MMA, 4 split, 4 epilogue
constexpr int kStages = 3;                    // ring of X / Xl tiles
constexpr int kSmemBytes = 1024 + 2 * kStages * kTile + 2 * kB + (3 * kStages + 4) * 8 + 16;
static_assert(kSmemBytes <= 227 * 1024, "shared memory per CTA");
constexpr uint32_t kWaitLimit = 1u << 22;     // bounded mbarrier waits
constexpr uint32_t kTmemCols = 128;           // two 128 x 64 FP32 accumulators

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait on an mbarrier phase; false after `limit` tries
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit = kWaitLimit) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 32) __nanosleep(64);
    }
    return false;
}

// Self-test of the timeout path: one thread waits on a fresh barrier that
// nothing arrives at, gives up after `limit` tries and records it in err.
__global__ void k_wait_selftest(int *err, uint32_t limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(b, 0, limit)) atomicExch(err, 1);
}

// AND of v over the 128 threads of the four epilogue warps (named barrier 1), so
// that they leave the loop together and their later barrier 1 syncs stay matched
__device__ __forceinline__ bool epilogue_all(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred p, 1, 128, q;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

// shared -> global tile store (bulk group of the issuing thread); rows beyond the
// tensor's extent are not written
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, uint32_t src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"((uint64_t)map),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row
// groups 1024 bytes apart (stride byte offset), leading byte offset unused.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                 // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major, M = 128, N = 64
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of element (row, col) in a K-major, 128-byte-swizzled tile with
// `rows` rows (two 128-byte K chunks of rows x 128 bytes)
__device__ __forceinline__ uint32_t swz_offset(int row, int col, int rows) {
    const int chunk = col >> 5, c = col & 31;
    return (uint32_t)(chunk * rows * 128 + row * 128 + ((((c >> 2) ^ (row & 7)) << 4) | ((c & 3) << 2)));
}

// Warp roles of the persistent kernel (one CTA per SM, tiles strided by the grid):
//   warp 0        TMA producer: tile i into ring stage i % kStages
//   warp 1        owns tensor memory; lane 0 issues the MMAs of tile i into
//                 accumulator i % 2 once the tile's low parts are written
//   warps 2..5    split: Xl = X - Xh for the stage
//   warps 6..9    epilogue: accumulator -> registers -> the stage's X buffer
//                 (same swizzled layout) -> the state, in place, by TMA store
// Barriers (all waits bounded): full[s] (TMA bytes landed), split[s] (the four
// split warps wrote Xl), empty[s] (the stage's result store has read it),
// accfull[a] (accumulator a holds a finished tile), accempty[a] (the epilogue
// read accumulator a).  Phase parities follow each barrier's use count.
__global__ void __launch_bounds__(kThreads, 1)
    k_block_tc(float *__restrict__ psi, const __grid_constant__ CUtensorMap tmap, const float *__restrict__ bh_g,
               const float *__restrict__ bl_g, uint64_t n_groups, uint64_t n_tiles, int *err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = smem;                          // kStages X tiles (the MMA reads them as Xh)
    unsigned char *sAl = smem + kStages * kTile;       // kStages Xl tiles
    unsigned char *sBh = smem + 2 * kStages * kTile;
    unsigned char *sBl = sBh + kB;
    uint64_t *bars = (uint64_t *)(sBl + kB);
    uint32_t *tmem_slot = (uint32_t *)(bars + 3 * kStages + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    auto bar = [&](int k) { return smem_u32(&bars[k]); };
    // barrier indices
    const int FULL = 0, SPLIT = kStages, EMPTY = 2 * kStages, ACCF = 3 * kStages, ACCE = 3 * kStages + 2;

    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) {
            mbar_init(bar(FULL + st), 1);
            mbar_init(bar(SPLIT + st), 4);
            mbar_init(bar(EMPTY + st), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(bar(ACCF + a), 1);
            mbar_init(bar(ACCE + a), 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // Bh, Bl: 64 x 64 row-major (row = output column n, col = k) into the swizzled layout
    for (int e = tid; e < kCols * kCols; e += kThreads) {
        const int n = e >> 6, k = e & 63;
        *(float *)(sBh + swz_offset(n, k, kCols)) = bh_g[e];
        *(float *)(sBl + swz_offset(n, k, kCols)) = bl_g[e];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // tiles of this CTA: blockIdx.x, blockIdx.x + gridDim.x, ...
    const uint64_t my_tiles = n_tiles > blockIdx.x ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            uint64_t issued = 0;
            for (uint64_t li = 0; li < my_tiles && ok; ++li) {
                const int st = (int)(li % kStages);
                const uint32_t use = (uint32_t)(li / kStages);
                if (li >= (uint64_t)kStages && !mbar_wait(bar(EMPTY + st), (use - 1) & 1u)) { ok = false; break; }
                const uint64_t tile = blockIdx.x + li * gridDim.x;
                mbar_expect_tx(bar(FULL + st), kTile);
                tma_load_2d(smem_u32(sA + st * kTile), &tmap, 0, (int)(tile * kRows), bar(FULL + st));
                tma_load_2d(smem_u32(sA + st * kTile + kChunk), &tmap, 32, (int)(tile * kRows), bar(FULL + st));
                ++issued;
            }
            // before leaving, wait (bounded) until the copies this thread issued
            // have landed, so that none writes shared memory after the CTA ends
            const uint64_t first = issued > (uint64_t)kStages ? issued - kStages : 0;
            for (uint64_t li = first; li < issued; ++li)
                if (!mbar_wait(bar(FULL + (int)(li % kStages)), (uint32_t)(li / kStages) & 1u)) ok = false;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            for (uint64_t li = 0; li < my_tiles && ok; ++li) {
                const int st = (int)(li % kStages), acc = (int)(li & 1);
                const uint32_t use = (uint32_t)(li / kStages), ause = (uint32_t)(li >> 1);
                if (!mbar_wait(bar(SPLIT + st), use & 1u)) { ok = false; break; }
                if (li >= 2 && !mbar_wait(bar(ACCE + acc), (ause - 1) & 1u)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned char *xa = sA + st * kTile, *xl = sAl + st * kTile;
                const unsigned char *As[3] = {xa, xa, xl};
                const unsigned char *Bs[3] = {sBh, sBl, sBh};
                const uint32_t d = tmem + (uint32_t)(acc * kCols);
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        const uint32_t koff = (uint32_t)((kk & 3) * 32);
                        const uint64_t a = smem_desc(smem_u32(As[p] + (kk >> 2) * kChunk) + koff);
                        const uint64_t b = smem_desc(smem_u32(Bs[p] + (kk >> 2) * kBChunk) + koff);
                        mma_tf32(d, a, b, (p | kk) ? 1u : 0u);
                    }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 bar(ACCF + acc))
                             : "memory");
            }
        }
    } else if (warp < 6) {
        const int sid = tid - 64;                      // 0..127
        for (uint64_t li = 0; li < my_tiles && ok; ++li) {
            const int st = (int)(li % kStages);
            if (!mbar_wait(bar(FULL + st), (uint32_t)(li / kStages) & 1u)) { ok = false; break; }
            const float4 *src = (const float4 *)(sA + st * kTile);
            float4 *dst = (float4 *)(sAl + st * kTile);
#pragma unroll 4
            for (int e = sid; e < kTile / 16; e += 128) {
                const float4 x = src[e];
                float4 l;
                l.x = x.x - __uint_as_float(__float_as_uint(x.x) & 0xFFFFE000u);
                l.y = x.y - __uint_as_float(__float_as_uint(x.y) & 0xFFFFE000u);
                l.z = x.z - __uint_as_float(__float_as_uint(x.z) & 0xFFFFE000u);
                l.w = x.w - __uint_as_float(__float_as_uint(x.w) & 0xFFFFE000u);
                dst[e] = l;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(SPLIT + st)) : "memory");
        }
    } else {
        const int quad = warp & 3;                     // TMEM lanes 32 quad .. 32 quad + 31
        const int r = quad * 32 + lane;                // tile row of this thread
        const bool leader = tid == 192;                // issues the stores (warp 6, lane 0)
        for (uint64_t li = 0; li < my_tiles && ok; ++li) {
            const int st = (int)(li % kStages), acc = (int)(li & 1);
            if (!epilogue_all(mbar_wait(bar(ACCF + acc), (uint32_t)(li >> 1) & 1u))) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float v0[32], v1[32];
            const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * kCols);
            tmem_ld32(taddr, v0);
            tmem_ld32(taddr + 32, v1);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(ACCE + acc)) : "memory");
            // the result row into the stage's X buffer (the products have read it)
            unsigned char *xs = sA + st * kTile;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                *(float4 *)(xs + swz_offset(r, 4 * q, kRows)) = make_float4(v0[4 * q], v0[4 * q + 1], v0[4 * q + 2], v0[4 * q + 3]);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                *(float4 *)(xs + swz_offset(r, 32 + 4 * q, kRows)) =
                    make_float4(v1[4 * q], v1[4 * q + 1], v1[4 * q + 2], v1[4 * q + 3]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("bar.sync 1, 128;" ::: "memory");    // the four epilogue warps
            if (leader) {
                const uint64_t tile = blockIdx.x + li * gridDim.x;
                tma_store_2d(&tmap, 0, (int)(tile * kRows), smem_u32(xs));
                tma_store_2d(&tmap, 32, (int)(tile * kRows), smem_u32(xs + kChunk));
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                // the stage goes back to the producer once the stores have read it
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(EMPTY + st)) : "memory");
            }
        }
        // every store complete before the CTA ends
        if (leader) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
    if (!ok) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

}  // namespace

cudaError_t launch_wait_selftest(int *err, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(err, 1u << 14);   // about a millisecond
    return cudaGetLastError();
}

cudaError_t launch_block_tc(void *psi, int n, const float *bh, const float *bl, int *err, int sms, cudaStream_t s) {
    if (n < 5) return cudaErrorInvalidValue;
    if (((uintptr_t)psi & 15) != 0) return cudaErrorInvalidValue;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const uint64_t n_groups = 1ull << (n - 5);
    CUtensorMap map;
    const cuuint64_t dims[2] = {64, (cuuint64_t)n_groups};
    const cuuint64_t strides[1] = {256};          // bytes between group rows
    const cuuint32_t box[2] = {32, (cuuint32_t)kRows};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, psi, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    // the shared-memory attribute is set once per device (host threads may launch
    // concurrently; setting it twice is harmless)
    static std::atomic<bool> attr_set[64];
    int dev = 0;
    cudaError_t ed = cudaGetDevice(&dev);
    if (ed != cudaSuccess) return ed;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev].load(std::memory_order_acquire)) {
        cudaError_t e = cudaFuncSetAttribute(k_block_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e != cudaSuccess) return e;
        attr_set[dev].store(true, std::memory_order_release);
    }
    const uint64_t n_tiles = (n_groups + kRows - 1) / kRows;
    uint64_t grid = n_tiles < (uint64_t)sms ? n_tiles : (uint64_t)sms;   // persistent: one CTA per SM
    k_block_tc<<<(unsigned)grid, kThreads, kSmemBytes, s>>>((float *)psi, map, bh, bl, n_groups, n_tiles, err);
    return cudaGetLastError();
}

}  // namespace qk
