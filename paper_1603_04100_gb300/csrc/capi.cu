// Status strings and version of the C ABI.
#include "common.cuh"

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
