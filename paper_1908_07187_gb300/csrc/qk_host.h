// Host-side helpers shared by the libqk translation units (no device code).
#pragma once

#include <cmath>
#include <complex>
#include <cstdint>

#include <cuda_runtime.h>

#include "qk.h"

namespace qk {

using cd = std::complex<double>;

// ---------------------------------------------------------------------------
// built-in gate matrices (textbook definitions; FP64)
// ---------------------------------------------------------------------------
// whether (id, p, np) names a built-in gate, and its target count, without
// forming the matrix (the same cases as builtin_matrix below)
inline bool builtin_arity(int id, const double *p, int np, int &ntargets) {
    ntargets = 1;
    switch (id) {
        case QK_GATE_X: case QK_GATE_Y: case QK_GATE_Z: case QK_GATE_H:
        case QK_GATE_S: case QK_GATE_SDG: case QK_GATE_T: case QK_GATE_TDG: return np == 0;
        case QK_GATE_U3: return np == 3 && p;
        case QK_GATE_P: case QK_GATE_RZ: return np == 1 && p;
        case QK_GATE_SWAP: ntargets = 2; return np == 0;
        default: return false;
    }
}

inline bool builtin_matrix(int id, const double *p, int np, cd m[4], int &ntargets) {
    const double r2 = 1.0 / std::sqrt(2.0);
    const cd I(0, 1);
    ntargets = 1;
    switch (id) {
        case QK_GATE_X: m[0] = 0; m[1] = 1; m[2] = 1; m[3] = 0; return np == 0;
        case QK_GATE_Y: m[0] = 0; m[1] = -I; m[2] = I; m[3] = 0; return np == 0;
        case QK_GATE_Z: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = -1; return np == 0;
        case QK_GATE_H: m[0] = r2; m[1] = r2; m[2] = r2; m[3] = -r2; return np == 0;
        case QK_GATE_S: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = I; return np == 0;
        case QK_GATE_SDG: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = -I; return np == 0;
        case QK_GATE_T: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = std::polar(1.0, M_PI / 4); return np == 0;
        case QK_GATE_TDG: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = std::polar(1.0, -M_PI / 4); return np == 0;
        case QK_GATE_U3: {
            if (np != 3 || !p) return false;
            const double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
            m[0] = c;
            m[1] = -std::polar(1.0, p[2]) * s;
            m[2] = std::polar(1.0, p[1]) * s;
            m[3] = std::polar(1.0, p[1] + p[2]) * c;
            return true;
        }
        case QK_GATE_P:
            if (np != 1 || !p) return false;
            m[0] = 1; m[1] = 0; m[2] = 0; m[3] = std::polar(1.0, p[0]);
            return true;
        case QK_GATE_RZ:
            if (np != 1 || !p) return false;
            m[0] = std::polar(1.0, -p[0] / 2); m[1] = 0; m[2] = 0; m[3] = std::polar(1.0, p[0] / 2);
            return true;
        case QK_GATE_SWAP: ntargets = 2; return np == 0;
        default: return false;
    }
}

// The library's stream-ordered device memory (contexts and batches) comes from
// one memory pool per device that keeps freed blocks for reuse.  A pool whose
// release threshold is 0 (the default pool's) hands freed memory back to the
// system at every stream or event synchronisation; with multi-GiB states that
// unmapping took up to ~0.2 s per synchronisation and stalled callers that free
// one state while others run.  Every context and batch holds the pool of its
// device from creation to destruction; when the last one on a device goes, the
// pool is trimmed back to empty.
// pool_acquire returns the pool (nullptr if it cannot be created: callers then
// use the device's default pool); pool_release drops one holder.
cudaMemPool_t pool_acquire(int device);
void pool_release(int device);
// stream-ordered allocation from the device's pool (or the default pool)
cudaError_t pool_malloc(void **p, size_t bytes, int device, cudaStream_t s);

// Inverse of a mod N by the extended Euclidean algorithm; ok = (gcd(a, N) == 1).
inline uint64_t modinv(uint64_t a, uint64_t N, bool &ok) {
    // extended Euclid on signed 128-bit
    __int128 t = 0, nt = 1, r = (__int128)N, nr = (__int128)(a % N);
    while (nr != 0) {
        __int128 q = r / nr, tmp;
        tmp = t - q * nt; t = nt; nt = tmp;
        tmp = r - q * nr; r = nr; nr = tmp;
    }
    ok = (r == 1);
    if (t < 0) t += N;
    return (uint64_t)t;
}

}  // namespace qk
