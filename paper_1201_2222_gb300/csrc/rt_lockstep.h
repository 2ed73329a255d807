// Lock-step Jacobi ALI solves of several grids on one stream, with the sweeps
// of compatible grids merged into shared launches (rt_api.cu).  Used by
// rt_ali_solve_many and by the request server's shared mode.
#pragma once

#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "rt_sc.h"

struct rt_lockstep_s;
typedef rt_lockstep_s *rt_lockstep;

struct LsResult {
  rt_grid g;
  void *tag;
  rt_status status;
  int iters;
  double resid;
  std::string message;   // the error message when status != RT_OK
};

rt_status ls_create(cudaStream_t s, rt_lockstep *out);
void ls_destroy(rt_lockstep L);
// Begins the solve of g (as rt_ali_solve with S = B would) and adds it.
// Errors: RT_ERR_STATE for a grid without medium, with the Gauss-Seidel
// iteration or with quadratic interpolation; RT_ERR_ARG for a negative tol.
rt_status ls_add(rt_lockstep L, rt_grid g, const rt_solve_opts *opts, void *tag);
// Iterates every member up to the nearest host check of one of them; members
// whose solve ended (converged, out of iterations or failed) are finished
// (their FP64 bins solved and merged) and moved to *done.  A CUDA error of
// the shared launches fails the call.
rt_status ls_step(rt_lockstep L, std::vector<LsResult> *done);
size_t ls_size(rt_lockstep L);
// Shared launches issued since the set was made or last reset (each sweeps
// several grids).
long long ls_shared_launches(rt_lockstep L);
void ls_reset_shared(rt_lockstep L);
