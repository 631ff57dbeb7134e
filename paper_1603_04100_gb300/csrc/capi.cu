// Status strings, version and the bounded-wait controls of the C ABI.
#include <atomic>

#include "common.cuh"

namespace mvgd {
namespace {
std::atomic<long long> g_wait_limit{0};  // 0: each kernel's own default
std::atomic<int> g_withhold{0};
std::atomic<int> g_solver_blocks{0};     // 0: as many as fit
std::atomic<int> g_stage_buffers{1};
std::atomic<int> g_assemble_warps{1};
}  // namespace

int tuned_solver_blocks_per_sm() { return g_solver_blocks.load(); }
int tuned_stage_buffers() { return g_stage_buffers.load(); }
int tuned_assemble_warps() { return g_assemble_warps.load(); }


long long wait_limit_or(long long dflt) {
    const long long v = g_wait_limit.load();
    return v > 0 ? v : dflt;
}

bool take_withhold() { return g_withhold.exchange(0) != 0; }
}  // namespace mvgd

MVGD_API const char* mvgd_status_string(mvgd_status s) {
    switch (s) {
        case MVGD_OK: return "MVGD_OK";
        case MVGD_EINVAL: return "MVGD_EINVAL: invalid argument";
        case MVGD_EWORKSPACE: return "MVGD_EWORKSPACE: workspace too small";
        case MVGD_EDEGENERATE: return "MVGD_EDEGENERATE: rank-deficient local fit";
        case MVGD_ENOCONV: return "MVGD_ENOCONV: iteration limit reached";
        case MVGD_EBREAKDOWN: return "MVGD_EBREAKDOWN: Krylov breakdown";
        case MVGD_ENONFINITE: return "MVGD_ENONFINITE: non-finite value";
        case MVGD_ECANCELLED: return "MVGD_ECANCELLED: cancelled";
        case MVGD_ETIMEOUT: return "MVGD_ETIMEOUT: device-side wait gave up";
        case MVGD_ECUDA: return "MVGD_ECUDA: CUDA runtime error";
        default: return "MVGD: unknown status";
    }
}

MVGD_API int32_t mvgd_version(void) { return 100; }

MVGD_API mvgd_status mvgd_set_wait_limit(int64_t polls) {
    if (polls < 0) return MVGD_EINVAL;
    mvgd::g_wait_limit.store((long long)polls);
    return MVGD_OK;
}

MVGD_API mvgd_status mvgd_test_withhold_arrival(int32_t on) {
    mvgd::g_withhold.store(on ? 1 : 0);
    return MVGD_OK;
}

MVGD_API mvgd_status mvgd_set_launch_tuning(int32_t solver_blocks_per_sm, int32_t stage_buffers,
                                            int32_t assemble_warps) {
    if (solver_blocks_per_sm < 0 || solver_blocks_per_sm > 32) return MVGD_EINVAL;
    if (stage_buffers < 0 || stage_buffers > 2) return MVGD_EINVAL;
    if (assemble_warps < 0 || assemble_warps > 8 || (assemble_warps & (assemble_warps - 1)) != 0) return MVGD_EINVAL;
    mvgd::g_solver_blocks.store(solver_blocks_per_sm);
    mvgd::g_stage_buffers.store(stage_buffers == 0 ? 1 : stage_buffers);
    mvgd::g_assemble_warps.store(assemble_warps == 0 ? 1 : assemble_warps);
    return MVGD_OK;
}
