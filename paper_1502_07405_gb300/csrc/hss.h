// HSS frontal matrices on the device (Section 4): randomized sampling by the
// skinny extend-add, Algorithm 1 with level-batched interpolative
// decompositions and the adaptive rank scheme, ULV-like factorization,
// low-rank Schur update, and their parts of the multifrontal solve.
#pragma once
#include "solver_ctx.h"

namespace hssmf {

hssmf_status hss_prepare(hssmf_ctx& c);       // host-side plan after analyze
hssmf_status hss_device_init(hssmf_ctx& c);   // device buffers at the first factor
void hss_release(hssmf_ctx& c);
void hss_begin_factor(hssmf_ctx& c);           // start of every numerical factorization
template <typename T>
hssmf_status hss_factor_level(hssmf_ctx& c, int level);
template <typename T>
hssmf_status hss_solve_fwd_level(hssmf_ctx& c, int level, T* W, int nrhs, int transpose);
template <typename T>
hssmf_status hss_solve_bwd_level(hssmf_ctx& c, int level, T* W, T* xp, int nrhs, int transpose);

}  // namespace hssmf
