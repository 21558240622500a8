// Emulator network kernels (placeholder).
#include "../../include/beor.h"
extern "C" {
int beor_mlp_create(beor_mlp** out, int, int, int, int, uint64_t) { if (out) *out = nullptr; return BEOR_ENOTSUP; }
int beor_mlp_destroy(beor_mlp*) { return BEOR_ENOTSUP; }
int beor_mlp_set_norm(beor_mlp*, const float*, const float*, float, float) { return BEOR_ENOTSUP; }
int beor_mlp_train_step(beor_mlp*, const float*, const float*, int, float, float, float, float, float*, void*) { return BEOR_ENOTSUP; }
int beor_mlp_infer(beor_mlp*, const float*, int, float*, void*) { return BEOR_ENOTSUP; }
int beor_mlp_get_params(beor_mlp*, int, float*, float*) { return BEOR_ENOTSUP; }
int beor_mlp_set_params(beor_mlp*, int, const float*, const float*) { return BEOR_ENOTSUP; }
int beor_mlp_grad(beor_mlp*, const float*, const float*, int, int, float*, float*, float*) { return BEOR_ENOTSUP; }
}
