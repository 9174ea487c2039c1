// Fused-mode queue entries and the planner interface (host only).
#pragma once

#include <complex>
#include <cstdint>
#include <functional>
#include <vector>

#include <cuda_runtime.h>

#include "qk.h"
#include "qk_kernels.cuh"

namespace qk {

// A queued unitary op in physical qubits.  U2: 2x2 matrix m on bit q where all
// cmask bits are 1.  PHASE: multiply amplitudes with (i & mask) == val by f.
struct FusedOp {
    enum Kind { U2 = 0, PHASE = 1 } kind = U2;
    int q = 0;
    uint64_t cmask = 0;
    std::complex<double> m[4];
    uint64_t mask = 0, val = 0;
    std::complex<double> f = 1.0;
    Cond cond{};
};

struct TilePlanner;
TilePlanner *make_planner();
void free_planner(TilePlanner *p);
// Plan an n-qubit (n >= 13) complex64 op list into tile passes; each pass's
// program goes to sink in order (the sink may adjust it before launching it).
// On a planner error *err names it.
using PassSink = std::function<qk_status(TileParams &)>;
qk_status plan_passes(TilePlanner *p, int n, const std::vector<FusedOp> &ops, const PassSink &sink, const char **err);
// plan_passes with each pass launched on the context's stream (n < 13 or
// complex128: one plain launch per op)
qk_status run_fused(TilePlanner *p, qk_ctx *c, const std::vector<FusedOp> &ops);

// context hooks implemented in qk_api.cu
void *ctx_state(qk_ctx *c);
int ctx_n(qk_ctx *c);
int ctx_prec(qk_ctx *c);
int ctx_sms(qk_ctx *c);
int ctx_tile_qubits(qk_ctx *c);
cudaStream_t ctx_stream(qk_ctx *c);
const uint8_t *ctx_cbits(qk_ctx *c);
qk_status ctx_run_plain(qk_ctx *c, const FusedOp &op);
qk_status ctx_fail(qk_ctx *c, qk_status s, const char *msg);
void ctx_launch_begin(qk_ctx *c, int cls, double bytes, void **token);
void ctx_launch_end(void *token);

}  // namespace qk
