// Generic-N integrator instantiations and the precision/size dispatch of the
// integrator.
#include "integrate_generic.cuh"
#include "integrate_grp.cuh"

// Parameter-set slots per warp of the lane-group kernel beyond the number
// that covers every group once (a tuning knob of the build).
#ifndef GRINS_GRP_SLOT_EXTRA
#define GRINS_GRP_SLOT_EXTRA 1
#endif

namespace grins {

cudaError_t launch_integrate_grp2(const IntegrateArgs &a, cudaStream_t st, int num_sms);
cudaError_t launch_integrate_grp4(const IntegrateArgs &a, cudaStream_t st, int num_sms);
cudaError_t launch_integrate_grp6(const IntegrateArgs &a, cudaStream_t st, int num_sms);
cudaError_t launch_integrate_grp8(const IntegrateArgs &a, cudaStream_t st, int num_sms);
cudaError_t launch_integrate_grp12(const IntegrateArgs &a, cudaStream_t st, int num_sms);

cudaError_t launch_integrate_fp32(const IntegrateArgs &a, cudaStream_t st, int num_sms)
{
    // the Tsitouras pair exists only in the kernels compiled for the network
    if (a.method != 0) return a.grp_jit ? launch_grp_jit(a.grp_jit, a, st, num_sms) : cudaErrorNotSupported;
    // lane-group kernel when the network has a layout and its slots fit in
    // shared memory; the generic kernel otherwise
    // (a layout with continuation rows is only for the register-record kernel)
    bool links = false;
    for (int r = 0; r < a.grp.R && r < kGrpMaxRows; ++r) links = links || a.grp.link_to[r] >= 0;
    if (a.grp.L > 0 && a.grp.R <= 12 && links) {
        if (a.grp_jit) {
            const cudaError_t e = launch_grp_jit(a.grp_jit, a, st, num_sms);
            if (e != cudaErrorInvalidConfiguration) return e;
        }
        return launch_dp5_generic<float>(a, st, num_sms);
    }
    if (a.grp.L > 0 && a.grp.R <= 12) {
        IntegrateArgs b = a;
        const int ndom = grp_domains(a.grp.L);               // scheduling domains per warp
        const int groups = kWarp / a.grp.L / ndom;           // groups per domain
        int s = (groups + a.n_ics - 1) / a.n_ics + GRINS_GRP_SLOT_EXTRA;
        s = s < 1 ? 1 : (s > 16 ? 16 : s);
        b.slots = s * ndom;
        cudaError_t e;
        if (a.grp_jit) {
            e = launch_grp_jit(a.grp_jit, b, st, num_sms);
            if (e != cudaErrorInvalidConfiguration) return e;
        }
        if (a.grp.R <= 2) e = launch_integrate_grp2(b, st, num_sms);
        else if (a.grp.R <= 4) e = launch_integrate_grp4(b, st, num_sms);
        else if (a.grp.R <= 6) e = launch_integrate_grp6(b, st, num_sms);
        else if (a.grp.R <= 8) e = launch_integrate_grp8(b, st, num_sms);
        else e = launch_integrate_grp12(b, st, num_sms);
        if (e != cudaErrorInvalidConfiguration) return e;
    }
    return launch_dp5_generic<float>(a, st, num_sms);
}

cudaError_t launch_integrate_fp64(const IntegrateArgs &a, cudaStream_t st, int num_sms)
{
    if (a.method != 0) return a.grp_jit ? launch_grp_jit(a.grp_jit, a, st, num_sms) : cudaErrorNotSupported;
    // the FP64 register-record kernel compiled for this network when there
    // is one; the generic kernel otherwise
    if (a.grp_jit) {
        const cudaError_t e = launch_grp_jit(a.grp_jit, a, st, num_sms);
        if (e != cudaErrorInvalidConfiguration) return e;
    }
    return launch_dp5_generic<double>(a, st, num_sms);
}

}  // namespace grins
