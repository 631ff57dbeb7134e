// Status strings, version and the bounded-wait controls of the C ABI.
#include <atomic>

#include "common.cuh"

namespace mvgd {
namespace {
std::atomic<long long> g_wait_limit{0};  // 0: each kernel's own default
std::atomic<int> g_withhold{0};
}  // namespace

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
