// Library-internal GP entry points (not part of the C ABI).
#pragma once
#include "mdgp.h"

// Factor the covariance of X only: posterior variances (Eq. predVarEq) need
// no outputs, so no alpha solve and no evidence terms are computed.
// mdgp_gp_predict on the handle fills the variances and sets every mean to
// the prior mean (mu_Xs, or 0).  Freed with mdgp_gp_free.
int gp_fit_variance_only(mdgp_ctx* ctx, const double* X, int64_t M, int32_t D, const mdgp_gp_params* params,
                         mdgp_gp** out);
