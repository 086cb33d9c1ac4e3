// Solver drivers (fitting, ALS, Rayleigh-Ritz, LOBPCG): placeholders until implemented.
#include "internal.h"

extern "C" {

ttn_status ttn_recompress(ttn_ctx* ctx, int, const double*, const ttn_ttno* const*,
                          const ttn_block* const*, const int*, ttn_block*, int, int,
                          ttn_precision) {
  if (ctx) ctx->last_error = "ttn_recompress: not built yet";
  return TTN_EUNSUPPORTED;
}
ttn_status ttn_als_solve(ttn_ctx* ctx, const ttn_ttno*, const double*, const ttn_block*,
                         ttn_block*, int, int, double, ttn_precision) {
  if (ctx) ctx->last_error = "ttn_als_solve: not built yet";
  return TTN_EUNSUPPORTED;
}
ttn_status ttn_rayleigh_ritz(ttn_ctx* ctx, int, const double*, const double*, int, double,
                             double*, double*) {
  if (ctx) ctx->last_error = "ttn_rayleigh_ritz: not built yet";
  return TTN_EUNSUPPORTED;
}
ttn_status ttn_lobpcg(ttn_ctx* ctx, const ttn_ttno*, ttn_block*, int, double, int, int, double,
                      int, ttn_precision, double*) {
  if (ctx) ctx->last_error = "ttn_lobpcg: not built yet";
  return TTN_EUNSUPPORTED;
}

}  // extern "C"
