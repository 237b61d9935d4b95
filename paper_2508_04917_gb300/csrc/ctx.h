// Host-side context object behind the opaque ilu0dd_ctx of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "internal.h"
#include "kernels.h"

using namespace ilu0dd;

struct ilu0dd_ctx {
  Plan plan;
  DevCtx dev{};
  unsigned char* ws = nullptr;
  size_t ws_bytes = 0;
  int device = 0;
  cudaStream_t own = nullptr;       // private stream of bicgstab_solve
  cudaGraphExec_t graph = nullptr;  // opts.check_every iterations
  int graph_iters = 0;
  double rtol = 1e-8;
  int32_t maxit = 10000;
  int check_every = 8;
  bool use_graphs = true;
  bool trace = false;
  double setup_s = 0.0;
  int last_iterations = 0;
  cudaError_t last_cuda = cudaSuccess;
  std::string why;
  std::vector<cudaEvent_t> events;  // bicgstab_iterate timing
  // ilu0_dd_apply_host: one stream per chunk of subdomains, and its events
  std::vector<cudaStream_t> hstreams;
  std::vector<cudaEvent_t> hevents;  // [0] caller's stream, [1 + i] chunk i done
  // host copies for ilu0_dd_export (opts.keep_host)
  std::vector<double> F, invD;
  bool have_factors = false;
};

// Host-side plan object behind the opaque ilu0dd_plan of the C ABI.
struct ilu0dd_plan {
  Plan plan;
  ilu0dd_opts opts{};
  std::string why;
  size_t scratch_bytes = 0;
  double t0 = 0.0;        // start of planning (setup time counts from here)
  bool consumed = false;  // moved into a context by ilu0_dd_setup_planned
};
