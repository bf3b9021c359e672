// mixed.cu -- MIXED32 particle half (placeholder until the tiled kernels land).
#include "mixed.h"

namespace pic {

struct MixedState {
    int unused;
};

int mixed_create(MixedState** out, const pic_params&, GridDev&, const GridDev*, long long, float*,
                 float*, CgState*, DevStatus*, std::string& err) {
    *out = nullptr;
    err = "PIC_MIXED32 is not available in this build";
    return PIC_EINVAL;
}
void mixed_destroy(MixedState* m) { delete m; }
int mixed_load(MixedState*, int, const double*, const double*, const double*, const double*,
               const double*, long long, cudaStream_t, std::string& err) {
    err = "PIC_MIXED32 is not available in this build";
    return PIC_EINVAL;
}
void mixed_enqueue_step(MixedState*, cudaStream_t) {}
int mixed_before_steps(MixedState*, cudaStream_t, std::string&) { return PIC_OK; }
int mixed_after_steps(MixedState*, cudaStream_t, std::string&) { return PIC_OK; }
long long mixed_count(MixedState*, int) { return 0; }
long long mixed_rebins(MixedState*) { return 0; }
int mixed_particles(MixedState*, int, double*, long long, cudaStream_t, std::string& err) {
    err = "PIC_MIXED32 is not available in this build";
    return PIC_EINVAL;
}

}  // namespace pic
