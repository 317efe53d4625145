// Definition of the library context (shared by the C-ABI translation units).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "device.h"

namespace pavg_detail {

using EventPair = std::pair<cudaEvent_t, cudaEvent_t>;

struct AvgPlan {
  double T = 0;
  int M = 0;                 // shifts in the plan (m1 - m0)
  int M_rule = 0;            // points of the quadrature rule the shifts come from
  int m0 = 0;                // first shift of the rule in the plan
  int K = 0;                 // K_max over shifts
  double* dA = nullptr;      // [M][K+1]  forward combine
  double* dB = nullptr;      // [K+1][M]  backward combine
  int* dlimA = nullptr;      // per 8-row tile of A: number of k with a nonzero entry
  int* dlimB = nullptr;      // per 8-row tile of B: number of (reordered) shifts with a nonzero entry
  // shifts in +s / -s pairs with equal coefficients and weights (symmetric
  // rules): the paired contractions replace dA / dB (then null)
  int P = 0;                 // pairs (0: not paired)
  double* dAp = nullptr;     // [P][K+1] c_k of each pair
  double* dBp = nullptr;     // [K+1][P] w c_k of each pair
  int* dlimAp = nullptr;     // per 8-pair tile: number of k with a nonzero entry
  int* dlimBp = nullptr;     // per 8-row tile: number of pairs with a nonzero entry
  cudaGraphExec_t exec = nullptr;
  bool timed = false;        // captured with CG event brackets
  int launches = 0;          // kernels in the captured graph
  std::vector<EventPair> pairs;   // CG event brackets inside the graph (owned)
};

// Mesh and operator data shared by the contexts with the same refinement,
// radius, rotation rate, device and geometry degree (reference counted,
// read-only after set-up).
using MeshKey = std::tuple<int, double, double, int, int>;
struct SharedMesh {
  int refs = 0;
  MeshKey key;
  pavg_detail::SharedMesh* shared = nullptr;
  pavg::Mesh mesh;
  pavg::DeviceMesh dm;  // topo stays per context
  // subdomain solver: the spectrum estimate (per mesh) and the partitions
  // built so far, by number of parts (P = 0 in a descriptor: not available)
  double sd_lmin = 0, sd_lmax = 0;
  std::vector<int32_t> tri;            // [F][4] DOF triples (host copy, for later partitions)
  std::map<int, pavg::SdMesh> sds;
};

}  // namespace pavg_detail

struct pavg_ctx {
  uint64_t uid = 0;  // unique per context in this process (a freed context's address can be reused)
  using AvgPlan = pavg_detail::AvgPlan;
  using EventPair = pavg_detail::EventPair;
  pavg_params p{};
  pavg_detail::SharedMesh* shared = nullptr;
  pavg::Mesh mesh;
  pavg::DeviceMesh dm;
  pavg::CgWork cg;
  pavg::CgParams cgp{};
  pavg::CgIrWork cgi;
  pavg::CgIrParams cgip{};
  pavg::SdMesh sd;              // the shared mesh's partition (copy of the descriptor)
  pavg::SdWork sdw;
  pavg::SdParams sdp{};
  bool use_sd = false;          // subdomain solver in use
  double lam = 0;
  int device = 0;
  // scratch
  double* ru = nullptr;         // [n_u] assembled velocity rhs
  double* facets = nullptr;     // [facet_chunk][F][3][15] facet terms of N per (cell, local edge)
  int facet_chunk = 1;          // states per N launch pair: kFacetChunk, fewer on large meshes
  double* vec[6] = {};          // [n] general vectors
  double* io_in = nullptr;      // [n] graph input
  double* io_out = nullptr;     // [n] graph output
  double* Q = nullptr;          // [(Kcap+1)][n] Chebyshev basis / backward coefficient vectors
  double* Um = nullptr;         // [Mcap][n] shifted states
  double* Rm = nullptr;         // [Mcap][n] weak-form N of the shifted states
  int Kcap = -1, Mcap = 0;
  double* ts = nullptr;         // [7][n] Lawson RK4 stage vectors, allocated by the first pavg_timestep
  double* host_part = nullptr;
  double* dpart = nullptr;
  cudaStream_t cap_stream = nullptr;
  std::map<std::tuple<double, int, int, int>, AvgPlan> plans;  // (T, M, m0, m1)
  int last_degree = 0;
  bool use_graphs = true;
  std::string err;
  // measurement: kernel launches and CG event brackets of the current / last call
  int launches = 0, last_launches = 0;
  bool timing = false;
  AvgPlan* capturing = nullptr;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<EventPair> cur_pairs, last_pairs;
};

