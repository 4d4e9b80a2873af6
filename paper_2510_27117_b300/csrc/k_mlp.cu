// k_mlp.cu -- learned proposal (placeholder entry points; kernels follow).
#include "internal.cuh"

extern "C" int64_t gfors_mlp_nparams(int32_t F, int32_t H) {
  if (F <= 0 || H <= 0) return 0;
  return (int64_t)H * F + H + (int64_t)H * H + H + H + 1;
}

cudaError_t gf_launch_features(GfCtx* h) { (void)h; return cudaErrorNotSupported; }
cudaError_t gf_launch_mlp_proposal(GfCtx* h) { (void)h; return cudaErrorNotSupported; }

extern "C" gfors_status gfors_set_proposal(gfors_handle h, const float* W, int64_t nW) {
  (void)W; (void)nW;
  return gf_fail(h, GFORS_E_UNSUPPORTED, "learned proposal not built yet");
}
extern "C" gfors_status gfors_get_features(gfors_handle h, int32_t inst, float* feat) {
  (void)inst; (void)feat;
  return gf_fail(h, GFORS_E_UNSUPPORTED, "learned proposal not built yet");
}
extern "C" gfors_status gfors_mlp_forward(int32_t, int32_t, const float*, int64_t, const float*,
                                          float*, float*, void*) {
  return GFORS_E_UNSUPPORTED;
}
extern "C" gfors_status gfors_mlp_loss_grad(int32_t, int32_t, const float*, int64_t,
                                            const float*, const float*, float*, double*, void*) {
  return GFORS_E_UNSUPPORTED;
}
extern "C" gfors_status gfors_mlp_adam(int64_t, float*, const float*, float*, float*, int64_t,
                                       double, double, double, double, void*) {
  return GFORS_E_UNSUPPORTED;
}
