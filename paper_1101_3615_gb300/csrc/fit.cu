// Symbol-expansion fit and preconditioner (placeholder until the FFT path lands).
#include "internal.h"

extern "C" probe_status probe_fit(probe_t h, const probe_basis* basis, const float* y, const float* Hy, int p,
                                  double* coeffs, double* resid_rel, probe_stream_t stream) {
    (void)h; (void)basis; (void)y; (void)Hy; (void)p; (void)coeffs; (void)resid_rel; (void)stream;
    return PROBE_ERR_STATE;
}

extern "C" probe_status probe_apply_precond(probe_t h, const probe_basis* basis, const double* coeffs,
                                            const float* img, float* out, probe_stream_t stream) {
    (void)h; (void)basis; (void)coeffs; (void)img; (void)out; (void)stream;
    return PROBE_ERR_STATE;
}
