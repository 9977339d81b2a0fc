// HSS fronts on the device: placeholder until the HSS kernels land.
#include "hss.h"

namespace hssmf {

struct HssState {};

hssmf_status hss_prepare(hssmf_ctx& c) {
  if (c.n_hss > 0) return c.fail(HSSMF_ERR_ARG, "HSS fronts are not available in this build");
  return HSSMF_OK;
}
hssmf_status hss_device_init(hssmf_ctx&) { return HSSMF_OK; }
void hss_release(hssmf_ctx& c) { c.hss = nullptr; }
template <typename T>
hssmf_status hss_factor_level(hssmf_ctx& c, int) { return c.fail(HSSMF_ERR_ARG, "no HSS"); }
template <typename T>
hssmf_status hss_solve_fwd_level(hssmf_ctx& c, int, T*, int, int) { return c.fail(HSSMF_ERR_ARG, "no HSS"); }
template <typename T>
hssmf_status hss_solve_bwd_level(hssmf_ctx& c, int, T*, T*, int, int) { return c.fail(HSSMF_ERR_ARG, "no HSS"); }

template hssmf_status hss_factor_level<double>(hssmf_ctx&, int);
template hssmf_status hss_factor_level<float>(hssmf_ctx&, int);
template hssmf_status hss_solve_fwd_level<double>(hssmf_ctx&, int, double*, int, int);
template hssmf_status hss_solve_fwd_level<float>(hssmf_ctx&, int, float*, int, int);
template hssmf_status hss_solve_bwd_level<double>(hssmf_ctx&, int, double*, double*, int, int);
template hssmf_status hss_solve_bwd_level<float>(hssmf_ctx&, int, float*, float*, int, int);

}  // namespace hssmf
