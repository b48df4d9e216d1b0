// The serving engine's per-request solve (engine.cu), driven by the serving
// loop (server.cu): Alg. 4 advanced one outer iteration at a time, with the
// filter's Clenshaw steps handed out as descriptors so that the steps of many
// requests run in one launch.
#pragma once
#include <memory>

#include "solver.h"
#include "spmm_multi.cuh"

namespace apf {

// One admitted request's solve.  The calls of one outer iteration, in order:
// begin_iteration (filter inputs on the request's stream), then for each
// global step g from max_steps - 1 down to 0 the descriptor of step g when
// g < steps() (batched() requests only), end_iteration (combine, orthogonalise,
// Rayleigh-Ritz, copy the Ritz values out: all on the request's stream), and
// check (synchronise, index sets, locking, next degree).
class EngineSolve {
 public:
  virtual ~EngineSolve() = default;
  virtual void begin_iteration() = 0;
  virtual bool batched() const = 0;     // filter steps go to the batched launch
  virtual bool is_complex() const = 0;
  virtual int steps() const = 0;        // Clenshaw steps of this iteration's recurrence
  virtual void step_desc(int g, MultiDesc* d) = 0;
  virtual void end_iteration() = 0;
  virtual void check() = 0;
  virtual bool finished() const = 0;
  // the result (ownership passes to the caller); status APF_OK or APF_ERR_NO_CONVERGENCE
  virtual apf_result* take_result(apf_status* status) = 0;
  apf_ctx* ctx = nullptr;
};

// Set-up of Alg. 4 for a request (bounds, coefficients, subspace size, the
// orthonormal initial block) on ctx's stream; throws ApfError.
std::unique_ptr<EngineSolve> engine_start(apf_ctx* ctx, const apf_matrix* A, const apf_params* prm);

// One batched Clenshaw step for the descriptors in a (real or complex FP32).
void engine_step_launch(apf_ctx* ctx, bool cplx, MultiArgs& a);

}  // namespace apf
