// C ABI of the pose-graph problem (include/ba.h, "Pose-graph optimisation";
// Sec. IV-D, Eqs. 3-4): the problem object, its device buffers and the LM
// trial as a sequence of stream-ordered launches, the PCG in one
// cooperative launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "ba.h"
#include "ba_internal.h"
#include "ba_pgo.cuh"

using namespace ba;

namespace {

#define PCU(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return set_error(e_ == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA, "%s failed: %s (%s:%d)", \
                       #call, cudaGetErrorString(e_), __FILE__, __LINE__);                     \
  } while (0)

inline unsigned nb(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// Per-incidence code from the stable sort of the 2E incidence keys
// [ei..., ej...]: 2 e for an edge's first node, 2 e + 1 for its second.
__global__ void k_pgo_inc_codes(int E, const int32_t* __restrict__ perm, const int32_t* __restrict__ ei,
                                const int32_t* __restrict__ ej, int32_t* __restrict__ inc, int2* __restrict__ inc2) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= 2 * E) return;
  const int k = perm[s];
  const int e = k < E ? k : k - E;
  inc[s] = k < E ? 2 * e : 2 * e + 1;
  inc2[s] = make_int2(e, k < E ? ej[e] : ei[e]);  // (edge, the other node)
}

// (t, q) [N][7] -> pose buffer [N][8] with a unit quaternion, qw >= 0; sets
// err bit 1 for a non-finite value or a zero quaternion.
__global__ void k_pgo_pack(int N, const double* __restrict__ in, double* __restrict__ out, int* __restrict__ err) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double v[7];
  bool ok = true;
  for (int k = 0; k < 7; ++k) {
    v[k] = in[7LL * n + k];
    ok = ok && isfinite(v[k]);
  }
  const double qq = v[3] * v[3] + v[4] * v[4] + v[5] * v[5] + v[6] * v[6];
  if (!ok || !(qq > 0.0)) {
    atomicOr(err, 2);
    v[3] = v[4] = v[5] = 0.0;
    v[6] = 1.0;
  }
  Pose P;
  for (int k = 0; k < 3; ++k) P.t[k] = v[k];
  for (int k = 0; k < 4; ++k) P.q[k] = v[3 + k];
  quat_normalise(P.q);
  store_pose(out + 8LL * n, P);
}

__global__ void k_pgo_unpack(int N, const double* __restrict__ in, double* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  for (int k = 0; k < 7; ++k) out[7LL * n + k] = in[8LL * n + k];
}

// Edge checks: indices in range and distinct, finite information matrices
// (err bits 0 and 1).
__global__ void k_pgo_check_edges(int N, int E, const int32_t* __restrict__ ei, const int32_t* __restrict__ ej,
                                  const double* __restrict__ info, int* __restrict__ err) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int i = ei[e], j = ej[e];
  if (i < 0 || i >= N || j < 0 || j >= N || i == j) atomicOr(err, 1);
  for (int k = 0; k < 21; ++k)
    if (!isfinite(info[21LL * e + k])) atomicOr(err, 2);
}

// y = (H + D) x over the free rows (x read as 0 at fixed nodes, y = 0 there);
// the product of the PCG's phase A with beta = 0.
__global__ void __launch_bounds__(PGO_PCG_THREADS)
k_pgo_matvec(int N, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ inc,
             const int32_t* __restrict__ ei, const int32_t* __restrict__ ej, const double* __restrict__ B,
             const double* __restrict__ D, const uint8_t* __restrict__ fixed, const double* __restrict__ x,
             double* __restrict__ y) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 6LL * N) return;
  const int n = (int)(t / 6), row = (int)(t % 6);
  auto xv = [&](int m, int k) { return (fixed && fixed[m]) ? 0.0 : x[6LL * m + k]; };
  double qa = 0.0;
  if (!(fixed && fixed[n])) {
    double xi[6];
    for (int k = 0; k < 6; ++k) xi[k] = xv(n, k);
    qa = D[t] * xi[row];
    const int end = rowptr[n + 1];
    for (int s = rowptr[n]; s < end; ++s) {
      const int code = inc[s];
      const int e = code >> 1;
      const int other = (code & 1) ? ei[e] : ej[e];
      const double* Br = B + 36LL * e + 6 * row;
      double acc = 0.0;
      for (int k = 0; k < 6; ++k) acc += Br[k] * (xi[k] - xv(other, k));
      qa += acc;
    }
  }
  y[t] = qa;
}

// SE(3) exponential applied to given poses (synthetic inputs):
// meas_e = Exp(noise_e) zeta_i^{-1} zeta_j, init_n = Exp(drift_n) zeta_n.
__global__ void k_pgo_synth(int N, int E, const double* __restrict__ gt, const int32_t* __restrict__ ei,
                            const int32_t* __restrict__ ej, const double* __restrict__ noise,
                            const double* __restrict__ drift, double* __restrict__ meas, double* __restrict__ init) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  auto pose = [&](int n) {
    Pose P;
    for (int a = 0; a < 3; ++a) P.t[a] = gt[7LL * n + a];
    for (int a = 0; a < 4; ++a) P.q[a] = gt[7LL * n + 3 + a];
    quat_normalise(P.q);
    return P;
  };
  auto put = [&](double* o, const Pose& P) {
    for (int a = 0; a < 3; ++a) o[a] = P.t[a];
    for (int a = 0; a < 4; ++a) o[3 + a] = P.q[a];
  };
  if (k < E) {
    const Pose Pi = pose(ei[k]), Pj = pose(ej[k]);
    // zeta_i^{-1} zeta_j = (R_i^T R_j, R_i^T (t_j - t_i))
    Pose rel;
    const double qic[4] = {-Pi.q[0], -Pi.q[1], -Pi.q[2], Pi.q[3]};
    quat_mul(qic, Pj.q, rel.q);
    double Ri[9];
    quat_rot(Pi.q, Ri);
    const double d[3] = {Pj.t[0] - Pi.t[0], Pj.t[1] - Pi.t[1], Pj.t[2] - Pi.t[2]};
    mat3T_vec(Ri, d, rel.t);
    double nz[6];
    for (int a = 0; a < 6; ++a) nz[a] = noise[6LL * k + a];
    put(meas + 7LL * k, retract(rel, nz));
  }
  if (k < N && init) {
    double dr[6];
    for (int a = 0; a < 6; ++a) dr[a] = drift[6LL * k + a];
    put(init + 7LL * k, retract(pose(k), dr));
  }
}

}  // namespace

struct ba_pgo {
  int N = 0, E = 0;
  ba_options opt{};
  int nbe = 0, nbn = 0;  // blocks of the edge and node kernels
  int pcg_grid = 0, pcg_npb = 0;  // PCG: blocks, nodes per block pass
  size_t pcg_res_smem = 0;        // > 0: the register-resident PCG, its shared memory
  int band = 0;                   // half-bandwidth of H + D in unknowns, in the factored order
  int32_t* pos = nullptr;         // Cholesky: block position of each node (RCM), or NULL (node order)
  double *rp = nullptr, *xp = nullptr;  // right-hand side and solution in the factored order
  std::vector<void*> allocs;
  int32_t *ei = nullptr, *ej = nullptr, *rowptr = nullptr, *inc = nullptr;
  int2* inc2 = nullptr;
  double *meas = nullptr, *info = nullptr, *poses = nullptr;
  double *B = nullptr, *qv = nullptr, *Hd = nullptr, *g = nullptr, *D = nullptr, *Minv = nullptr;
  double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  double *pcg_part = nullptr, *dpart = nullptr, *gpart = nullptr, *epart = nullptr;
  uint8_t* fixed = nullptr;
  // Cholesky: the band tiles of H + D (then L), 1 / L_cc, the inverses
  // L_JJ^{-T}, y / x in the padded factored order, and the flags of the
  // factorisation's schedule (tile final and tile updates [bnb (bwt + 1)]
  // each, counters [5], failure [1], inverse final [bnb])
  int bnb = 0, bwt = 0, band_grid = 0, band_crit = 0, bntask = 0, bncrit = 0;
  size_t bT_bytes = 0, bflag_count = 0;
  double *bT = nullptr, *brs = nullptr, *bUi = nullptr, *dy = nullptr;
  int* bflag = nullptr;
  int4* btask = nullptr;  // the factorisation's tasks in ticket order
  int* derr = nullptr;
  GridBar* bar = nullptr;
  DevState* st = nullptr;
  ba_iter_stats* stats = nullptr;

  template <typename P>
  cudaError_t alloc(P** ptr, size_t bytes) {
    void* v = nullptr;
    const cudaError_t e = cudaMalloc(&v, bytes ? bytes : 16);
    if (e == cudaSuccess) {
      allocs.push_back(v);
      *ptr = reinterpret_cast<P*>(v);
    }
    return e;
  }
  ~ba_pgo() {
    for (void* v : allocs) cudaFree(v);
  }
};

namespace {

ba_status copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  PCU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
  return BA_OK;
}


// Reverse Cuthill-McKee order of the pose graph (the factored order of the
// Cholesky solver): per connected component, a pseudo-peripheral start
// (the lowest-degree node of the last breadth-first level, twice), then a
// breadth-first walk visiting each node's unvisited neighbours by
// increasing degree (ties by index), reversed.  Returns order[k] = the node
// at position k.
std::vector<int32_t> rcm_order(int N, const std::vector<int32_t>& ei, const std::vector<int32_t>& ej) {
  std::vector<std::vector<int32_t>> adj(N);
  for (size_t k = 0; k < ei.size(); ++k) {
    adj[ei[k]].push_back(ej[k]);
    adj[ej[k]].push_back(ei[k]);
  }
  std::vector<int32_t> deg(N);
  for (int i = 0; i < N; ++i) {
    std::sort(adj[i].begin(), adj[i].end());
    adj[i].erase(std::unique(adj[i].begin(), adj[i].end()), adj[i].end());
    deg[i] = (int32_t)adj[i].size();
  }
  std::vector<char> done(N, 0);
  std::vector<int32_t> level(N, -1), order, touched, q;
  order.reserve(N);
  // breadth-first levels from s within the unplaced nodes; returns the last
  // level's lowest-degree node and the eccentricity
  auto far_node = [&](int s0, int& ecc) {
    for (int v : touched) level[v] = -1;
    touched.clear();
    q.assign(1, s0);
    level[s0] = 0;
    touched.push_back(s0);
    for (size_t h = 0; h < q.size(); ++h)
      for (int w : adj[q[h]])
        if (!done[w] && level[w] < 0) {
          level[w] = level[q[h]] + 1;
          touched.push_back(w);
          q.push_back(w);
        }
    ecc = level[q.back()];
    int best = q.back();
    for (int v : q)
      if (level[v] == ecc && (deg[v] < deg[best] || (deg[v] == deg[best] && v < best))) best = v;
    return best;
  };
  for (;;) {
    int start = -1;
    for (int i = 0; i < N; ++i)
      if (!done[i] && (start < 0 || deg[i] < deg[start])) start = i;
    if (start < 0) break;
    int ecc = 0;
    int cand = far_node(start, ecc);
    for (int rep = 0; rep < 2; ++rep) {
      int e2 = 0;
      const int c2 = far_node(cand, e2);
      if (e2 <= ecc) break;
      start = cand;
      cand = c2;
      ecc = e2;
    }
    start = cand;
    // Cuthill-McKee walk of the component
    q.assign(1, start);
    done[start] = 1;
    std::vector<int32_t> nb;
    for (size_t h = 0; h < q.size(); ++h) {
      const int v = q[h];
      order.push_back(v);
      nb.clear();
      for (int w : adj[v])
        if (!done[w]) nb.push_back(w);
      std::sort(nb.begin(), nb.end(), [&](int a, int b) { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; });
      for (int w : nb) {
        done[w] = 1;
        q.push_back(w);
      }
    }
  }
  std::reverse(order.begin(), order.end());
  return order;
}

ba_status check_pgo_options(const ba_options* o) {
  if (o->precision != BA_PREC_F64) return set_error(BA_ERR_INVALID_ARG, "pose graphs run in FP64 (BA_PREC_F64)");
  if (!(o->lambda0 > 0) || !(o->up > 1) || !(o->down > 0 && o->down < 1) || !(o->lambda_min > 0) ||
      !(o->lambda_max >= o->lambda_min) || !(o->diag_min >= 0) || !(o->diag_max >= o->diag_min))
    return set_error(BA_ERR_INVALID_ARG, "damping options out of range");
  if (o->pcg_maxiter < 0 || o->pcg_maxiter > 1000000 || !(o->pcg_tol >= 0))
    return set_error(BA_ERR_INVALID_ARG, "pcg_maxiter must be in [0, 1000000] and pcg_tol >= 0");
  if (o->max_stats < 1 || o->max_stats > (1 << 24)) return set_error(BA_ERR_INVALID_ARG, "max_stats out of range");
  if (o->huber_delta != 0.0) return set_error(BA_ERR_INVALID_ARG, "pose graphs take no robust loss");
  if (o->solver != BA_SOLVER_PCG && o->solver != BA_SOLVER_CHOLESKY)
    return set_error(BA_ERR_INVALID_ARG, "solver must be BA_SOLVER_PCG or BA_SOLVER_CHOLESKY");
  return BA_OK;
}

// Read st->err and the barrier flag; a set bit becomes the call's error.
ba_status check_device_errors(ba_pgo* h, cudaStream_t s) {
  PCU(cudaStreamSynchronize(s));
  int herr = 0;
  GridBar gb{};
  PCU(cudaMemcpy(&herr, h->derr, sizeof(int), cudaMemcpyDeviceToHost));
  PCU(cudaMemcpy(&gb, h->bar, sizeof(GridBar), cudaMemcpyDeviceToHost));
  if (gb.err) return set_error(BA_ERR_TIMEOUT, "a PCG grid barrier wait ran out");
  if (herr & 1) return set_error(BA_ERR_INVALID_ARG, "an edge index is out of range or joins a node to itself");
  if (herr & 2) return set_error(BA_ERR_NONFINITE, "a non-finite pose, measurement or information entry");
  return BA_OK;
}

void enqueue_cost(ba_pgo* h, cudaStream_t s) {
  k_pgo_edge_cost<<<h->nbe, PGO_EDGE_THREADS, 0, s>>>(h->E, h->ei, h->ej, h->meas, h->info, h->poses, h->N, h->st,
                                                      0, nullptr, nullptr, h->epart);
  k_pgo_cost_set<<<1, 256, 0, s>>>(h->nbe, h->epart, h->st);
  count_launch(2);
}

void enqueue_lin(ba_pgo* h, int force, double* r_out, double* A_out, cudaStream_t s) {
  k_pgo_lin<<<h->nbe, PGO_EDGE_THREADS, 0, s>>>(h->E, h->ei, h->ej, h->meas, h->info, h->poses, h->N, h->st, force,
                                                h->B, h->qv, r_out, A_out);
  k_pgo_node<<<h->nbn, PGO_NODE_THREADS, 0, s>>>(h->N, h->rowptr, h->inc, h->B, h->qv, h->st, force, h->Hd, h->g);
  count_launch(2);
}

ba_status enqueue_solve(ba_pgo* h, const double* lam_ptr, int maxiter, double tol, cudaStream_t s) {
  k_pgo_damp<<<h->nbn, PGO_NODE_THREADS, 0, s>>>(h->N, h->Hd, h->g, h->fixed, lam_ptr, h->opt.diag_min,
                                                 h->opt.diag_max, h->D, h->Minv, h->x, h->r, h->dpart, h->st);
  count_launch();
  if (h->opt.solver == BA_SOLVER_CHOLESKY) {
    // H + D is banded in the factored order (node order, or a reverse
    // Cuthill-McKee order when that is narrower; half-bandwidth h->band):
    // its band tiles are assembled, then factored and solved in one
    // cooperative launch (ba_band.cuh)
    const int n = 6 * h->N;
    PCU(cudaMemsetAsync(h->bT, 0, h->bT_bytes, s));
    PCU(cudaMemsetAsync(h->bflag, 0, sizeof(int) * h->bflag_count, s));
    k_pgo_band<<<h->N, 64, 0, s>>>(h->N, h->rowptr, h->inc, h->ei, h->ej, h->B, h->Hd, h->D, h->pos, h->fixed,
                                   h->bwt, h->bT);
    count_launch();
    if (h->bnb * BAND_TB > n) {
      k_band_pad<<<1, BAND_TB, 0, s>>>(n, h->bnb, h->bwt, h->bT);
      count_launch();
    }
    const double* rhs = h->r;
    double* sol = h->x;
    if (h->pos) {
      k_pgo_permute<<<nb(n, 256), 256, 0, s>>>(h->N, h->pos, 0, h->r, h->rp);
      count_launch();
      rhs = h->rp;
      sol = h->xp;
    }
    const size_t ntile = (size_t)h->bnb * (h->bwt + 1);
    int* ctr = h->bflag + 2 * ntile;
    BandArgs ba_{h->bnb, h->bwt, n, h->bntask, h->bncrit, h->band_crit, h->btask, h->bT, h->brs, h->bUi, rhs,
                 h->dy, sol, h->bflag, h->bflag + ntile, ctr, ctr + 5, ctr + 6};
    void* args[] = {&ba_};
    PCU(cudaLaunchCooperativeKernel((const void*)k_band_chol, dim3(h->band_grid), dim3(BAND_THREADS), args, 0, s));
    k_band_finish<<<nb(n, 256), 256, 0, s>>>(n, ctr + 5, ctr, sol, h->st);
    count_launch(2);
    if (h->pos) {
      k_pgo_permute<<<nb(n, 256), 256, 0, s>>>(h->N, h->pos, 1, h->xp, h->x);
      count_launch();
    }
    return BA_OK;
  }
  PCU(cudaMemsetAsync(h->bar, 0, sizeof(GridBar), s));
  PcgArgs a;
  a.N = h->N;
  a.npb = h->pcg_npb;
  a.rowptr = h->rowptr;
  a.inc2 = h->inc2;
  a.B = h->B;
  a.D = h->D;
  a.Minv = h->Minv;
  a.fixed = h->fixed;
  a.x = h->x;
  a.r = h->r;
  a.z = h->z;
  a.p = h->p;
  a.q = h->q;
  a.part = h->pcg_part;
  a.bpart = h->dpart;
  a.nbp = h->nbn;
  a.maxiter = maxiter;
  a.tol = tol;
  a.bar = h->bar;
  a.st = h->st;
  void* args[] = {&a};
  if (h->pcg_res_smem)
    PCU(cudaLaunchCooperativeKernel((const void*)k_pgo_pcg_res, dim3(h->pcg_grid), dim3(6 * h->pcg_npb), args,
                                    h->pcg_res_smem, s));
  else
    PCU(cudaLaunchCooperativeKernel((const void*)k_pgo_pcg, dim3(h->pcg_grid), dim3(6 * h->pcg_npb), args, 0, s));
  count_launch();
  return BA_OK;
}

ba_status enqueue_trial(ba_pgo* h, cudaStream_t s) {
  enqueue_lin(h, 0, nullptr, nullptr, s);
  ba_status e = enqueue_solve(h, &h->st->lam, h->opt.pcg_maxiter, h->opt.pcg_tol, s);
  if (e != BA_OK) return e;
  k_pgo_trial<<<h->nbn, PGO_NODE_THREADS, 0, s>>>(h->N, h->x, h->g, h->fixed, h->poses, h->st, h->gpart);
  k_pgo_edge_cost<<<h->nbe, PGO_EDGE_THREADS, 0, s>>>(h->E, h->ei, h->ej, h->meas, h->info, h->poses, h->N, h->st,
                                                      1, h->x, h->B, h->epart);
  const ba_options& o = h->opt;
  k_pgo_control<<<1, 256, 0, s>>>(h->nbe, h->epart, h->nbn, h->gpart, h->nbn, h->dpart, o.up, o.down, o.rho_good,
                                  o.rho_bad, o.lambda_min, o.lambda_max, h->st, h->stats, o.max_stats);
  count_launch(3);
  return BA_OK;
}

ba_status out_copy(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (!dst) return BA_OK;
  PCU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
  return BA_OK;
}

}  // namespace

extern "C" {

ba_status ba_pgo_create(ba_pgo** out, int N, int E, const double* poses, const int32_t* ei, const int32_t* ej,
                        const double* meas, const double* info, const uint8_t* fixed, const ba_options* opt,
                        void* stream) {
  if (!out) return set_error(BA_ERR_INVALID_ARG, "NULL output handle");
  *out = nullptr;
  if (N < 2 || E < 1 || 2LL * E > (1LL << 30))
    return set_error(BA_ERR_INVALID_ARG, "need N >= 2 nodes and 1 <= E < 2^29 edges");
  if (!poses || !ei || !ej || !meas || !info) return set_error(BA_ERR_INVALID_ARG, "NULL input array");
  ba_options o;
  if (opt) o = *opt;
  else ba_options_default(&o);
  ba_status st = check_pgo_options(&o);
  if (st != BA_OK) return st;
  int dev = 0, coop = 0, nsm = 0, occ = 0;
  PCU(cudaGetDevice(&dev));
  PCU(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  PCU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (!coop) return set_error(BA_ERR_CUDA, "the device does not support cooperative launches");
  // PCG: about one block per SM, npb consecutive nodes per block pass
  const int npb = std::max(1, std::min(PGO_PCG_NODES, (N + nsm - 1) / nsm));
  PCU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pgo_pcg, 6 * npb, 0));
  if (occ < 1) return set_error(BA_ERR_CUDA, "the PCG kernel cannot be resident");
  ba_pgo* h = new (std::nothrow) ba_pgo();
  if (!h) return set_error(BA_ERR_OOM, "host allocation failed");
  auto bail = [&](ba_status e) {
    delete h;
    return e;
  };
  h->N = N;
  h->E = E;
  h->opt = o;
  h->nbe = nb(E, PGO_EDGE_THREADS);
  h->nbn = nb(N, PGO_NODE_THREADS);
  const int groups = (N + npb - 1) / npb;
  h->pcg_npb = npb;
  h->pcg_grid = std::max(1, std::min(groups, occ * nsm));
  cudaStream_t s = (cudaStream_t)stream;
  const long long n6 = 6LL * N;
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t bytes) {
    if (e == cudaSuccess) e = h->alloc(p, bytes);
  };
  A(&h->ei, 4ull * E);
  A(&h->ej, 4ull * E);
  A(&h->rowptr, 4ull * (N + 1));
  A(&h->inc, 8ull * E);
  A(&h->inc2, 16ull * E);
  A(&h->meas, 64ull * E);
  A(&h->info, 168ull * E);
  A(&h->poses, 128ull * N);
  A(&h->B, 288ull * E);
  A(&h->qv, 48ull * E);
  A(&h->Hd, 168ull * N);
  A(&h->g, 8ull * n6);
  A(&h->D, 8ull * n6);
  A(&h->Minv, 288ull * N);
  A(&h->x, 8ull * n6);
  A(&h->r, 8ull * n6);
  A(&h->z, 8ull * n6);
  A(&h->p, 16ull * n6);
  A(&h->q, 8ull * n6);
  A(&h->pcg_part, 32ull * h->pcg_grid);
  A(&h->dpart, 16ull * h->nbn);
  A(&h->gpart, 8ull * h->nbn);
  A(&h->epart, 16ull * h->nbe);
  A(&h->derr, sizeof(int));
  A(&h->bar, sizeof(GridBar));
  A(&h->st, sizeof(DevState));
  A(&h->stats, sizeof(ba_iter_stats) * (size_t)o.max_stats);
  if (fixed) A(&h->fixed, (size_t)N);
  std::vector<int32_t> hpos;  // Cholesky: block position of each node, empty for the node order
  int32_t* keys = nullptr;
  int32_t* perm = nullptr;
  void* scratch = nullptr;
  double* tmp7 = nullptr;
  A(&keys, 8ull * E);
  A(&perm, 8ull * E);
  A(&scratch, csr_scratch_bytes(2 * E));
  A(&tmp7, 56ull * std::max(N, E));
  if (e != cudaSuccess) return bail(set_error(e == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA,
                                              "device allocation failed: %s", cudaGetErrorString(e)));
  if ((st = copy_in(h->ei, ei, 4ull * E, s)) != BA_OK) return bail(st);
  if ((st = copy_in(h->ej, ej, 4ull * E, s)) != BA_OK) return bail(st);
  if ((st = copy_in(h->info, info, 168ull * E, s)) != BA_OK) return bail(st);
  if ((e = cudaMemsetAsync(h->derr, 0, sizeof(int), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(h->bar, 0, sizeof(GridBar), s)) != cudaSuccess)
    return bail(set_error(BA_ERR_CUDA, "memset failed"));
  // the edges are checked before any kernel indexes with them
  k_pgo_check_edges<<<h->nbe, PGO_EDGE_THREADS, 0, s>>>(N, E, h->ei, h->ej, h->info, h->derr);
  count_launch();
  if ((st = check_device_errors(h, s)) != BA_OK) return bail(st);
  {
    // half-bandwidth of H in the node order: 6 max |i - j| + 5 unknowns
    std::vector<int32_t> hi(E), hj(E);
    if ((e = cudaMemcpy(hi.data(), h->ei, 4ull * E, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(hj.data(), h->ej, 4ull * E, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return bail(set_error(BA_ERR_CUDA, "copy of the edges failed"));
    long long bwn = 0;
    for (int k = 0; k < E; ++k) bwn = std::max<long long>(bwn, std::llabs((long long)hi[k] - hj[k]));
    h->band = (int)std::min<long long>(6 * bwn + 5, n6 - 1);
    if (o.solver == BA_SOLVER_CHOLESKY) {
      // the reverse Cuthill-McKee order when its band is narrower
      const std::vector<int32_t> order = rcm_order(N, hi, hj);
      hpos.assign(N, 0);
      for (int k = 0; k < N; ++k) hpos[order[k]] = k;
      long long bwr = 0;
      for (int k = 0; k < E; ++k) bwr = std::max<long long>(bwr, std::llabs((long long)hpos[hi[k]] - hpos[hj[k]]));
      if (bwr < bwn) {
        h->band = (int)std::min<long long>(6 * bwr + 5, n6 - 1);
        if ((e = h->alloc(&h->pos, 4ull * N)) != cudaSuccess || (e = h->alloc(&h->rp, 8ull * n6)) != cudaSuccess ||
            (e = h->alloc(&h->xp, 8ull * n6)) != cudaSuccess ||
            (e = cudaMemcpy(h->pos, hpos.data(), 4ull * N, cudaMemcpyHostToDevice)) != cudaSuccess)
          return bail(set_error(e == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA, "reordering set-up failed"));
      } else {
        hpos.clear();  // node order
      }
      // the band tiles and the schedule's flags
      h->bnb = (int)((n6 + BAND_TB - 1) / BAND_TB);
      h->bwt = std::min(h->bnb - 1, (h->band + BAND_TB - 1) / BAND_TB);
      // updates per task segment: one column, or more when the band is so
      // wide that the task list would pass 4M updates
      const long long nupd = (long long)h->bnb * h->bwt * (h->bwt + 1) / 2;
      if (nupd > (1LL << 40))
        return bail(set_error(BA_ERR_INVALID_ARG, "the band of H is too wide for BA_SOLVER_CHOLESKY (%d x %d tiles)",
                              h->bnb, h->bwt + 1));
      const int s_upd = (int)std::max(1LL, (nupd + (4LL << 20) - 1) / (4LL << 20));
      // one block per SM: a task then has its SM's FP64 pipe to itself
      h->band_grid = std::max(1, nsm);
      h->band_crit = h->band_grid >= 2 ? std::min(BAND_CRIT_BLOCKS, std::max(1, h->band_grid / 8)) : 0;
      const std::vector<BandTask> tasks = band_tasks(h->bnb, h->bwt, s_upd, h->band_grid, h->band_crit, &h->bncrit);
      static_assert(sizeof(BandTask) == sizeof(int4), "a task is read as an int4");
      if (h->bncrit == 0) h->band_crit = 0;
      h->bntask = (int)tasks.size();
      h->bT_bytes = (size_t)h->bnb * (h->bwt + 1) * (BAND_TB * BAND_TB) * sizeof(double);
      h->bflag_count = 2 * (size_t)h->bnb * (h->bwt + 1) + 6 + h->bnb;
      int occb = 0;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occb, k_band_chol, BAND_THREADS, 0)) != cudaSuccess ||
          occb < 1)
        return bail(set_error(BA_ERR_CUDA, "the Cholesky kernel cannot be resident"));
      if ((e = h->alloc(&h->bT, h->bT_bytes)) != cudaSuccess ||
          (e = h->alloc(&h->brs, 8ull * h->bnb * BAND_TB)) != cudaSuccess ||
          (e = h->alloc(&h->bUi, 8ull * h->bnb * BAND_TB * BAND_TB)) != cudaSuccess ||
          (e = h->alloc(&h->dy, 8ull * h->bnb * BAND_TB)) != cudaSuccess ||
          (e = h->alloc(&h->bflag, sizeof(int) * h->bflag_count)) != cudaSuccess ||
          (e = h->alloc(&h->btask, sizeof(int4) * tasks.size())) != cudaSuccess ||
          (e = cudaMemcpy(h->btask, tasks.data(), sizeof(int4) * tasks.size(), cudaMemcpyHostToDevice)) !=
              cudaSuccess)
        return bail(set_error(e == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA,
                              "allocation of the band (%zu bytes) failed", h->bT_bytes));
    }
  }
  // incidence CSR: stable sort of [ei..., ej...] by node
  if ((e = cudaMemcpyAsync(keys, h->ei, 4ull * E, cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(keys + E, h->ej, 4ull * E, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return bail(set_error(BA_ERR_CUDA, "copy failed"));
  if ((e = csr_build_async(keys, 2 * E, N, perm, h->rowptr, scratch, h->derr, s)) != cudaSuccess)
    return bail(set_error(BA_ERR_CUDA, "incidence sort failed: %s", cudaGetErrorString(e)));
  k_pgo_inc_codes<<<nb(2LL * E, 256), 256, 0, s>>>(E, perm, h->ei, h->ej, h->inc, h->inc2);
  count_launch();
  {
    // the register-resident PCG when every block can hold one node group
    // with its incidence slots in shared memory, all blocks resident
    std::vector<int32_t> rp(N + 1);
    if ((e = cudaMemcpyAsync(rp.data(), h->rowptr, 4ull * (N + 1), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return bail(set_error(BA_ERR_CUDA, "copy of the incidence rows failed"));
    int max_slots = 0;
    for (int g0 = 0; g0 < N; g0 += npb) max_slots = std::max(max_slots, rp[std::min(N, g0 + npb)] - rp[g0]);
    const size_t smem = pgo_res_smem(max_slots);
    int occ_res = 0;
    if (smem <= 200u * 1024u &&
        cudaFuncSetAttribute(k_pgo_pcg_res, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_res, k_pgo_pcg_res, 6 * npb, smem) == cudaSuccess &&
        groups <= (long long)occ_res * nsm) {
      h->pcg_res_smem = std::max<size_t>(smem, 16);
      h->pcg_grid = groups;
    }
    cudaGetLastError();
  }
  // poses and measurements, quaternions normalised
  if ((st = copy_in(tmp7, poses, 56ull * N, s)) != BA_OK) return bail(st);
  k_pgo_pack<<<nb(N, 128), 128, 0, s>>>(N, tmp7, h->poses, h->derr);
  if ((st = copy_in(tmp7, meas, 56ull * E, s)) != BA_OK) return bail(st);
  k_pgo_pack<<<nb(E, 128), 128, 0, s>>>(E, tmp7, h->meas, h->derr);
  count_launch(2);
  if (fixed) {
    if ((st = copy_in(h->fixed, fixed, (size_t)N, s)) != BA_OK) return bail(st);
  }
  {
    DevState init{};
    init.lam = o.lambda0;
    init.lam_probe = o.lambda0;
    init.need_lin = 1;
    init.need_cost = 1;
    if ((e = cudaMemcpyAsync(h->st, &init, sizeof(DevState), cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return bail(set_error(BA_ERR_CUDA, "state copy failed"));
  }
  enqueue_cost(h, s);
  if ((st = check_device_errors(h, s)) != BA_OK) return bail(st);
  DevState hs{};
  if ((e = cudaMemcpy(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return bail(set_error(BA_ERR_CUDA, "state copy failed"));
  if (!std::isfinite(hs.F)) return bail(set_error(BA_ERR_NONFINITE, "the initial cost is not finite"));
  *out = h;
  return BA_OK;
}

ba_status ba_pgo_destroy(ba_pgo* h) {
  delete h;
  return BA_OK;
}

ba_status ba_pgo_solve(ba_pgo* h, int iters, void* stream) {
  if (!h || iters < 0) return set_error(BA_ERR_INVALID_ARG, "NULL handle or negative iteration count");
  cudaStream_t s = (cudaStream_t)stream;
  for (int t = 0; t < iters; ++t) {
    const ba_status e = enqueue_trial(h, s);
    if (e != BA_OK) return e;
  }
  return check_device_errors(h, s);
}

ba_status ba_pgo_get_poses(ba_pgo* h, double* poses_out, void* stream) {
  if (!h || !poses_out) return set_error(BA_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  DevState hs{};
  PCU(cudaMemcpyAsync(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  PCU(cudaStreamSynchronize(s));
  double* tmp = h->p;  // scratch of 12N doubles: holds the [N][7] poses
  k_pgo_unpack<<<nb(h->N, 128), 128, 0, s>>>(h->N, h->poses + (long long)hs.cur * 8 * h->N, tmp);
  count_launch();
  PCU(cudaMemcpyAsync(poses_out, tmp, 56ull * h->N, cudaMemcpyDefault, s));
  PCU(cudaStreamSynchronize(s));
  return BA_OK;
}

ba_status ba_pgo_set_poses(ba_pgo* h, const double* poses, void* stream) {
  if (!h || !poses) return set_error(BA_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  DevState hs{};
  PCU(cudaMemcpyAsync(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  PCU(cudaStreamSynchronize(s));
  PCU(cudaMemcpyAsync(h->p, poses, 56ull * h->N, cudaMemcpyDefault, s));
  k_pgo_pack<<<nb(h->N, 128), 128, 0, s>>>(h->N, h->p, h->poses + (long long)hs.cur * 8 * h->N, h->derr);
  count_launch();
  const int one = 1;
  PCU(cudaMemcpyAsync(&h->st->need_lin, &one, sizeof(int), cudaMemcpyHostToDevice, s));
  enqueue_cost(h, s);
  return check_device_errors(h, s);
}

ba_status ba_pgo_get_stats(ba_pgo* h, ba_iter_stats* host_out, int cap, int* n_out) {
  if (!h || (!host_out && cap > 0) || cap < 0) return set_error(BA_ERR_INVALID_ARG, "bad arguments");
  PCU(cudaDeviceSynchronize());
  DevState hs{};
  PCU(cudaMemcpy(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost));
  const long long total = hs.trials;
  const long long ring = h->opt.max_stats;
  const long long avail = std::min(total, ring);
  const long long n = std::min<long long>(avail, cap);
  // the last n records, oldest first
  for (long long k = 0; k < n; ++k) {
    const long long t = total - n + k;
    PCU(cudaMemcpy(host_out + k, h->stats + (t % ring), sizeof(ba_iter_stats), cudaMemcpyDeviceToHost));
  }
  if (n_out) *n_out = (int)n;
  return BA_OK;
}

ba_status ba_pgo_get_scalars(ba_pgo* h, double* cost, double* lambda) {
  if (!h) return set_error(BA_ERR_INVALID_ARG, "NULL handle");
  PCU(cudaDeviceSynchronize());
  DevState hs{};
  PCU(cudaMemcpy(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost));
  if (cost) *cost = hs.F;
  if (lambda) *lambda = hs.lam;
  return BA_OK;
}

ba_status ba_pgo_set_lambda(ba_pgo* h, double lambda) {
  if (!h || !(lambda > 0)) return set_error(BA_ERR_INVALID_ARG, "NULL handle or lambda <= 0");
  PCU(cudaDeviceSynchronize());
  PCU(cudaMemcpy(&h->st->lam, &lambda, sizeof(double), cudaMemcpyHostToDevice));
  return BA_OK;
}

ba_status ba_pgo_linearize(ba_pgo* h, double* r, double* A, double* B, double* Hd, double* g, double* cost,
                           void* stream) {
  if (!h) return set_error(BA_ERR_INVALID_ARG, "NULL handle");
  cudaStream_t s = (cudaStream_t)stream;
  const long long E = h->E, N = h->N;
  // per-edge r and A go to scratch owned here, then out
  double* rr = nullptr;
  double* AA = nullptr;
  if (r) PCU(cudaMalloc((void**)&rr, 48ull * E));
  if (A && cudaMalloc((void**)&AA, 288ull * E) != cudaSuccess) {
    if (rr) cudaFree(rr);
    return set_error(BA_ERR_OOM, "scratch allocation failed");
  }
  enqueue_lin(h, 1, rr, AA, s);
  ba_status st = BA_OK;
  if (st == BA_OK && r) st = out_copy(r, rr, 48ull * E, s);
  if (st == BA_OK && A) st = out_copy(A, AA, 288ull * E, s);
  if (st == BA_OK) st = out_copy(B, h->B, 288ull * E, s);
  if (st == BA_OK) st = out_copy(Hd, h->Hd, 168ull * N, s);
  if (st == BA_OK) st = out_copy(g, h->g, 48ull * N, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && st == BA_OK) st = set_error(BA_ERR_CUDA, "linearisation failed");
  if (rr) cudaFree(rr);
  if (AA) cudaFree(AA);
  if (st != BA_OK) return st;
  if (cost) {
    DevState hs{};
    PCU(cudaMemcpy(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost));
    *cost = hs.F;
  }
  return check_device_errors(h, s);
}

ba_status ba_pgo_matvec(ba_pgo* h, double lambda, const double* x, double* y, void* stream) {
  if (!h || !x || !y || !(lambda >= 0)) return set_error(BA_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const long long n6 = 6LL * h->N;
  enqueue_lin(h, 0, nullptr, nullptr, s);
  PCU(cudaMemcpyAsync(&h->st->lam_probe, &lambda, sizeof(double), cudaMemcpyHostToDevice, s));
  k_pgo_damp<<<h->nbn, PGO_NODE_THREADS, 0, s>>>(h->N, h->Hd, h->g, h->fixed, &h->st->lam_probe, h->opt.diag_min,
                                                 h->opt.diag_max, h->D, h->Minv, h->x, h->r, h->dpart, h->st);
  PCU(cudaMemcpyAsync(h->z, x, 8ull * n6, cudaMemcpyDefault, s));
  k_pgo_matvec<<<nb(n6, PGO_PCG_THREADS), PGO_PCG_THREADS, 0, s>>>(h->N, h->rowptr, h->inc, h->ei, h->ej, h->B,
                                                                    h->D, h->fixed, h->z, h->q);
  count_launch(2);
  PCU(cudaMemcpyAsync(y, h->q, 8ull * n6, cudaMemcpyDefault, s));
  return check_device_errors(h, s);
}

ba_status ba_pgo_damped_solve(ba_pgo* h, double lambda, int maxiter, double tol, double* dx, int* iters,
                              double* rel, void* stream) {
  if (!h || !dx || !(lambda >= 0) || maxiter < 0 || !(tol >= 0)) return set_error(BA_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  enqueue_lin(h, 0, nullptr, nullptr, s);
  PCU(cudaMemcpyAsync(&h->st->lam_probe, &lambda, sizeof(double), cudaMemcpyHostToDevice, s));
  ba_status st = enqueue_solve(h, &h->st->lam_probe, maxiter, tol, s);
  if (st != BA_OK) return st;
  PCU(cudaMemcpyAsync(dx, h->x, 48ull * h->N, cudaMemcpyDefault, s));
  if ((st = check_device_errors(h, s)) != BA_OK) return st;
  DevState hs{};
  PCU(cudaMemcpy(&hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost));
  if (iters) *iters = hs.pcg_iters;
  if (rel) *rel = hs.pcg_rel;
  return BA_OK;
}

ba_status ba_pgo_synthesize(int N, int E, const double* poses_gt, const int32_t* ei, const int32_t* ej,
                            const double* noise, const double* drift, double* meas_out, double* init_out,
                            void* stream) {
  if (N < 1 || E < 0 || !poses_gt || (E > 0 && (!ei || !ej || !noise || !meas_out)) || (init_out && !drift))
    return set_error(BA_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  double *dg = nullptr, *dn = nullptr, *dd = nullptr, *dm = nullptr, *di = nullptr;
  int32_t *dei = nullptr, *dej = nullptr;
  auto cleanup = [&]() {
    for (void* v : {(void*)dg, (void*)dn, (void*)dd, (void*)dm, (void*)di, (void*)dei, (void*)dej})
      if (v) cudaFree(v);
  };
  cudaError_t e = cudaMalloc(&dg, 56ull * N);
  if (e == cudaSuccess && E > 0) e = cudaMalloc(&dn, 48ull * E);
  if (e == cudaSuccess && E > 0) e = cudaMalloc(&dm, 56ull * E);
  if (e == cudaSuccess && E > 0) e = cudaMalloc(&dei, 4ull * E);
  if (e == cudaSuccess && E > 0) e = cudaMalloc(&dej, 4ull * E);
  if (e == cudaSuccess && init_out) e = cudaMalloc(&dd, 48ull * N);
  if (e == cudaSuccess && init_out) e = cudaMalloc(&di, 56ull * N);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dg, poses_gt, 56ull * N, cudaMemcpyDefault, s);
  if (e == cudaSuccess && E > 0) e = cudaMemcpyAsync(dn, noise, 48ull * E, cudaMemcpyDefault, s);
  if (e == cudaSuccess && E > 0) e = cudaMemcpyAsync(dei, ei, 4ull * E, cudaMemcpyDefault, s);
  if (e == cudaSuccess && E > 0) e = cudaMemcpyAsync(dej, ej, 4ull * E, cudaMemcpyDefault, s);
  if (e == cudaSuccess && init_out) e = cudaMemcpyAsync(dd, drift, 48ull * N, cudaMemcpyDefault, s);
  if (e == cudaSuccess) {
    std::vector<int32_t> hi(E), hj(E);
    if (E > 0) {
      e = cudaMemcpyAsync(hi.data(), dei, 4ull * E, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(hj.data(), dej, 4ull * E, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      for (int k = 0; e == cudaSuccess && k < E; ++k)
        if (hi[k] < 0 || hi[k] >= N || hj[k] < 0 || hj[k] >= N) {
          cleanup();
          return set_error(BA_ERR_INVALID_ARG, "edge %d: node index out of range", k);
        }
    }
  }
  if (e == cudaSuccess) {
    k_pgo_synth<<<nb(std::max(N, E), 128), 128, 0, s>>>(N, E, dg, dei, dej, dn, dd, dm, di);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && E > 0) e = cudaMemcpyAsync(meas_out, dm, 56ull * E, cudaMemcpyDefault, s);
  if (e == cudaSuccess && init_out) e = cudaMemcpyAsync(init_out, di, 56ull * N, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) return set_error(BA_ERR_CUDA, "synthesis failed: %s", cudaGetErrorString(e));
  return BA_OK;
}

}  // extern "C"
