// C ABI of the batched form (include/ba.h, "Batched form"): many small
// independent LM problems solved by one persistent launch, its launch
// configuration and its autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <new>
#include <string>
#include <vector>

#include "ba.h"
#include "ba_batch.cuh"
#include "ba_internal.h"
#include "ba_kernels.cuh"
#include "ba_problem.h"

using namespace ba;

#define BA_BATCH_MAX_STATS 256
static_assert(BA_BATCH_MAX_CAMS == BMAXC, "header and kernel disagree on the cameras per problem");

struct ba_batch {
  ba_problem* h = nullptr;  // the concatenated problem (structure, buffers)
  int nprob = 0, cap = 0, nsm = 0;
  std::vector<int32_t> cam_off, pt_off, obs_off, chunk_off;
  int32_t *d_cam_off = nullptr, *d_pt_off = nullptr, *d_chunk_off = nullptr, *d_bchunk = nullptr,
          *d_order = nullptr;
  double* dot_gp = nullptr;
  BState* state = nullptr;
  BState* state0 = nullptr;  // the state every reset starts from
  ba_iter_stats* stats = nullptr;
  int* work = nullptr;
  void *cams0 = nullptr, *pts0 = nullptr;  // parameters at creation (internal order)
  // launch configuration
  int ctas_per_sm = 1, variant = 0, order = 0;
  // segment sizes: camera-major pieces of at most piece_max slots, point
  // chunks of at most chunk_slots slots and chunk_pts points
  int piece_max = PIECE, chunk_slots = CHUNK_SLOTS, chunk_pts = CHUNK_PTS;
  size_t piece_cap = 0, chunk_cap = 0;  // capacity of the piece and chunk arrays
  size_t smem = 0;
  // graph of one solve
  cudaGraphExec_t gexec = nullptr;
  int g_iters = -1, g_grid = -1, g_variant = -1;
  std::vector<void*> allocs;

  template <typename X>
  cudaError_t alloc(X** ptr, size_t bytes) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, bytes > 0 ? bytes : 16);
    if (e == cudaSuccess) {
      allocs.push_back(v);
      *ptr = static_cast<X*>(v);
    }
    return e;
  }
  ~ba_batch() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (h) ba_problem_destroy(h);
    for (void* v : allocs) cudaFree(v);
  }
};

namespace {

#define BCU(call)                                                                                  \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return set_error(e_ == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA, "%s failed: %s", \
                       #call, cudaGetErrorString(e_));                                             \
  } while (0)

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// Point chunks of each problem (runs of whole points with at most slots
// observations and pts points; a point with more observations is a chunk
// alone), the problems' ranges into b->chunk_off; rq: the point rows.
std::vector<int32_t> cut_chunks(ba_batch* b, const std::vector<int32_t>& rq, int slots, int pts) {
  std::vector<int32_t> bch;
  b->chunk_off.assign(b->nprob + 1, 0);
  for (int i = 0; i < b->nprob; ++i) {
    b->chunk_off[i] = (int32_t)bch.size();
    const int pend = b->pt_off[i + 1];
    long long j = b->pt_off[i];
    while (j < pend) {
      bch.push_back((int32_t)j);
      long long e = j + 1;
      while (e < pend && e - j < pts && rq[e + 1] - rq[j] <= slots) ++e;
      j = e;
    }
    bch.push_back(pend);
  }
  b->chunk_off[b->nprob] = (int32_t)bch.size();
  return bch;
}

ba_status enter(ba_batch* b, void* stream) {
  BCU(cudaEventRecord(b->h->ev_in, (cudaStream_t)stream));
  BCU(cudaStreamWaitEvent(b->h->s, b->h->ev_in, 0));
  return BA_OK;
}
ba_status leave(ba_batch* b, void* stream) {
  BCU(cudaEventRecord(b->h->ev_out, b->h->s));
  BCU(cudaStreamWaitEvent((cudaStream_t)stream, b->h->ev_out, 0));
  return BA_OK;
}

template <typename T>
BatchArgs<T> make_args(ba_batch* b, int iters) {
  ba_problem* h = b->h;
  const ba_options& o = h->opt;
  BatchArgs<T> a{};
  a.nprob = b->nprob;
  a.C = h->C;
  a.P = h->P;
  a.O = h->O;
  a.cam_off = b->d_cam_off;
  a.pt_off = b->d_pt_off;
  a.chunk_off = b->d_chunk_off;
  a.bchunk = b->d_bchunk;
  a.order = b->d_order;
  a.piece_cam = h->piece_cam;
  a.piece_beg = h->piece_beg;
  a.piece_end = h->piece_end;
  a.cam_piece_ptr = h->cam_piece_ptr;
  a.cm_pt = h->cm_pt;
  a.rowptr_pt = h->rowptr_pt;
  a.pm2cm = h->pm2cm;
  a.pm_cam = h->pm_cam;
  a.pm_pt = h->pm_pt;
  a.cm_px = (const T*)h->cm_px;
  a.pm_px = (const T*)h->pm_px;
  a.cams = (T*)h->cams;
  a.pts = (T*)h->pts;
  a.camtab = (T*)h->camtab;
  a.ptab = (T*)h->ptab;
  a.zbuf = (T*)h->zbuf;
  a.Jcm = (T*)h->Jcm;
  a.cm_sw = (T*)h->cm_sw;
  a.pm_sw = (T*)h->pm_sw;
  a.Vinv = (T*)h->Vinv;
  a.y0 = (T*)h->y0;
  a.dp = (T*)h->dp;
  a.V = h->V;
  a.gp = h->gp;
  a.part = h->part;
  a.dot_gp = b->dot_gp;
  a.state = b->state;
  a.stats = b->stats;
  a.cap = b->cap;
  a.work = b->work;
  a.iters = iters;
  a.delta = (T)(o.huber_delta > 0 ? o.huber_delta : 0.0);
  a.up = o.up;
  a.down = o.down;
  a.rho_good = o.rho_good;
  a.rho_bad = o.rho_bad;
  a.lam_min = o.lambda_min;
  a.lam_max = o.lambda_max;
  a.dmin = o.diag_min;
  a.dmax = o.diag_max;
  a.tol = o.pcg_tol;
  a.maxiter = o.pcg_maxiter;
  return a;
}

// The kernel instance for (T, MF, variant).
template <typename T, bool MF>
const void* kernel_for(int variant) {
  return variant == 1 ? (const void*)k_batch_lm<T, MF, 2> : (const void*)k_batch_lm<T, MF, 1>;
}

const void* kernel_of(const ba_batch* b, int variant) {
  const ba_problem* h = b->h;
  if (h->prec == BA_PREC_F32) return h->mf ? kernel_for<float, true>(variant) : kernel_for<float, false>(variant);
  return h->mf ? kernel_for<double, true>(variant) : kernel_for<double, false>(variant);
}

int grid_of(const ba_batch* b) { return std::max(1, std::min(b->nprob, b->ctas_per_sm * b->nsm)); }

template <typename T>
cudaError_t launch_solve(ba_batch* b, int iters, cudaStream_t s) {
  BatchArgs<T> a = make_args<T>(b, iters);
  cudaError_t e = cudaMemsetAsync(b->work, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  return cudaLaunchKernel(kernel_of(b, b->variant), dim3(grid_of(b)), dim3(BT), args, b->smem, s);
}

// Enqueue one solve: capture [work-list reset, persistent kernel] once per
// (iters, grid, variant) and replay the graph.
ba_status enqueue_solve(ba_batch* b, int iters) {
  ba_problem* h = b->h;
  const int grid = grid_of(b);
  if (!b->gexec || b->g_iters != iters || b->g_grid != grid || b->g_variant != b->variant) {
    if (b->gexec) {
      cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    BCU(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = h->prec == BA_PREC_F32 ? launch_solve<float>(b, iters, h->s) : launch_solve<double>(b, iters, h->s);
    cudaError_t e2 = cudaStreamEndCapture(h->s, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->gexec = nullptr;
      return set_error(BA_ERR_CUDA, "batched solve capture failed: %s", cudaGetErrorString(e));
    }
    b->g_iters = iters;
    b->g_grid = grid;
    b->g_variant = b->variant;
  }
  BCU(cudaGraphLaunch(b->gexec, h->s));
  count_launch(1);
  return BA_OK;
}

ba_status upload_order(ba_batch* b) {
  std::vector<int32_t> ord(b->nprob);
  for (int i = 0; i < b->nprob; ++i) ord[i] = i;
  if (b->order == 0) {
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
      return b->obs_off[x + 1] - b->obs_off[x] > b->obs_off[y + 1] - b->obs_off[y];
    });
  }
  BCU(cudaMemcpy(b->d_order, ord.data(), ord.size() * 4, cudaMemcpyHostToDevice));
  return BA_OK;
}

// Every problem back to its starting state (stream-ordered).
ba_status init_state(ba_batch* b) {
  BCU(cudaMemcpyAsync(b->state, b->state0, b->nprob * sizeof(BState), cudaMemcpyDeviceToDevice, b->h->s));
  BCU(cudaMemsetAsync(b->stats, 0, (size_t)b->nprob * b->cap * sizeof(ba_iter_stats), b->h->s));
  return BA_OK;
}

int occupancy(const ba_batch* b, int variant) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel_of(b, variant), BT, b->smem) != cudaSuccess) return 1;
  return std::max(1, n);
}

template <typename T, bool MF>
cudaError_t set_smem_attr(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_batch_lm<T, MF, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batch_lm<T, MF, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e;
}

std::string tune_key(const ba_batch* b) {
  cudaDeviceProp prop{};
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  std::string name = prop.name;
  for (char& ch : name)
    if (ch == '"' || ch == '\\' || ch == '|') ch = '_';
  const ba_problem* h = b->h;
  // histogram of problem sizes: observations per problem in powers of two
  int hist[32] = {0};
  for (int i = 0; i < b->nprob; ++i) {
    int o = b->obs_off[i + 1] - b->obs_off[i], k = 0;
    while (o > 1 && k < 31) {
      o >>= 1;
      ++k;
    }
    hist[k]++;
  }
  std::string key = name + "|" + (h->prec == BA_PREC_F32 ? "f32" : "f64") + (h->mf ? "-recompute" : "-store") +
                    "|pcg" + std::to_string(h->opt.pcg_maxiter) + "|n" + std::to_string(b->nprob) + "|h";
  for (int k = 0; k < 32; ++k)
    if (hist[k]) key += " " + std::to_string(k) + ":" + std::to_string(hist[k]);
  return key;
}

bool json_int(const std::string& line, const char* field, int* out) {
  const std::string pat = std::string("\"") + field + "\":";
  const size_t p = line.find(pat);
  if (p == std::string::npos) return false;
  *out = (int)strtol(line.c_str() + p + pat.size(), nullptr, 10);
  return true;
}

}  // namespace

extern "C" {

ba_status ba_batch_create(ba_batch** out, int nprob, const int32_t* cam_counts, const int32_t* pt_counts,
                          const int32_t* obs_counts, const void* cams, const void* points, const int32_t* cam_idx,
                          const int32_t* pt_idx, const void* pixels, const ba_options* opt, void* stream) {
  if (!out) return set_error(BA_ERR_INVALID_ARG, "NULL output handle");
  *out = nullptr;
  if (nprob < 1) return set_error(BA_ERR_INVALID_ARG, "nprob must be >= 1 (got %d)", nprob);
  if (!cam_counts || !pt_counts || !obs_counts || !cams || !points || !cam_idx || !pt_idx || !pixels)
    return set_error(BA_ERR_INVALID_ARG, "NULL input array");
  ba_batch* b = new (std::nothrow) ba_batch();
  if (!b) return set_error(BA_ERR_OOM, "host allocation failed");
  b->nprob = nprob;
  b->cam_off.assign(nprob + 1, 0);
  b->pt_off.assign(nprob + 1, 0);
  b->obs_off.assign(nprob + 1, 0);
  long long sc = 0, sp = 0, so = 0;
  for (int i = 0; i < nprob; ++i) {
    if (cam_counts[i] < 1 || cam_counts[i] > BA_BATCH_MAX_CAMS || pt_counts[i] < 1 || obs_counts[i] < 1) {
      delete b;
      return set_error(BA_ERR_INVALID_ARG, "problem %d: need 1 <= C_b <= %d, P_b >= 1, O_b >= 1 (got %d, %d, %d)",
                       i, BA_BATCH_MAX_CAMS, cam_counts[i], pt_counts[i], obs_counts[i]);
    }
    sc += cam_counts[i];
    sp += pt_counts[i];
    so += obs_counts[i];
    if (sc > INT32_MAX / 64 || sp > INT32_MAX / 8 || so > INT32_MAX / 32) {
      delete b;
      return set_error(BA_ERR_INVALID_ARG, "batch too large for int32 indexing");
    }
    b->cam_off[i + 1] = (int32_t)sc;
    b->pt_off[i + 1] = (int32_t)sp;
    b->obs_off[i + 1] = (int32_t)so;
  }
  const int C = (int)sc, P = (int)sp, O = (int)so;
  cudaStream_t s = (cudaStream_t)stream;
  ba_status st = BA_OK;
  {
    // global indices of the concatenated problem
    int32_t *gci = nullptr, *gpi = nullptr, *offs = nullptr;
    cudaError_t e = cudaMalloc(&gci, (size_t)O * 4);
    if (e == cudaSuccess) e = cudaMalloc(&gpi, (size_t)O * 4);
    if (e == cudaSuccess) e = cudaMalloc(&offs, 3ull * (nprob + 1) * 4);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(offs, b->obs_off.data(), (nprob + 1) * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(offs + (nprob + 1), b->cam_off.data(), (nprob + 1) * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(offs + 2 * (nprob + 1), b->pt_off.data(), (nprob + 1) * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      k_batch_globalize<<<nblk(O, 256), 256, 0, s>>>(O, nprob, offs, offs + (nprob + 1), offs + 2 * (nprob + 1),
                                                     cam_idx, pt_idx, gci, gpi);
      count_launch();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) st = ba_problem_create(&b->h, C, P, O, cams, points, gci, gpi, pixels, opt, stream);
    else st = set_error(e == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA, "batch set-up failed: %s",
                        cudaGetErrorString(e));
    cudaFree(gci);
    cudaFree(gpi);
    cudaFree(offs);
  }
  if (st != BA_OK) {
    delete b;
    return st;
  }
  ba_problem* h = b->h;
  auto fail_out = [&](ba_status code, const char* msg) {
    delete b;
    return set_error(code, "%s", msg);
  };
  // every point observed: then problem b's points keep the internal range
  // [pt_off[b], pt_off[b+1]) (points are renumbered by their first camera)
  std::vector<int32_t> rq(P + 1);
  if (cudaMemcpy(rq.data(), h->rowptr_pt, (P + 1) * 4ull, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail_out(BA_ERR_CUDA, "copy of the point rows failed");
  for (int j = 0; j < P; ++j)
    if (rq[j + 1] == rq[j]) return fail_out(BA_ERR_INVALID_ARG, "every point of a batched problem must be observed");
  // point chunks of each problem, cut as a problem of its own cuts them
  std::vector<int32_t> bch = cut_chunks(b, rq, CHUNK_SLOTS, CHUNK_PTS);
  b->chunk_cap = bch.size();
  b->piece_cap = (size_t)h->npieces;
  b->cap = std::min(h->opt.max_stats, BA_BATCH_MAX_STATS);
  const size_t ts = h->tsize;
  cudaError_t e = b->alloc(&b->d_cam_off, (nprob + 1) * 4ull);
  if (e == cudaSuccess) e = b->alloc(&b->d_pt_off, (nprob + 1) * 4ull);
  if (e == cudaSuccess) e = b->alloc(&b->d_chunk_off, (nprob + 1) * 4ull);
  if (e == cudaSuccess) e = b->alloc(&b->d_bchunk, bch.size() * 4);
  if (e == cudaSuccess) e = b->alloc(&b->d_order, nprob * 4ull);
  if (e == cudaSuccess) e = b->alloc(&b->dot_gp, bch.size() * 8);
  if (e == cudaSuccess) e = b->alloc(&b->state, nprob * sizeof(BState));
  if (e == cudaSuccess) e = b->alloc(&b->state0, nprob * sizeof(BState));
  if (e == cudaSuccess) e = b->alloc(&b->stats, (size_t)nprob * b->cap * sizeof(ba_iter_stats));
  if (e == cudaSuccess) e = b->alloc(&b->work, sizeof(int));
  if (e == cudaSuccess) e = b->alloc(&b->cams0, 9ull * C * ts);
  if (e == cudaSuccess) e = b->alloc(&b->pts0, 3ull * P * ts);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_cam_off, b->cam_off.data(), (nprob + 1) * 4ull, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_pt_off, b->pt_off.data(), (nprob + 1) * 4ull, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_chunk_off, b->chunk_off.data(), (nprob + 1) * 4ull, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_bchunk, bch.data(), bch.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->cams0, h->cams, 9ull * C * ts, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->pts0, h->pts, 3ull * P * ts, cudaMemcpyDeviceToDevice);
  {
    std::vector<BState> st0(nprob);
    for (auto& x : st0) {
      x = BState{};
      x.lam = h->opt.lambda0;
      x.need_cost = 1;
    }
    if (e == cudaSuccess) e = cudaMemcpy(b->state0, st0.data(), nprob * sizeof(BState), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess)
    return fail_out(e == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA, "batch allocation failed");
  b->smem = h->prec == BA_PREC_F32 ? sizeof(BShared<float>) : sizeof(BShared<double>);
  if (h->prec == BA_PREC_F32) e = h->mf ? set_smem_attr<float, true>(b->smem) : set_smem_attr<float, false>(b->smem);
  else e = h->mf ? set_smem_attr<double, true>(b->smem) : set_smem_attr<double, false>(b->smem);
  int dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail_out(BA_ERR_CUDA, "kernel attribute set-up failed");
  b->variant = 0;
  b->ctas_per_sm = occupancy(b, 0);
  b->order = 0;
  st = upload_order(b);
  if (st == BA_OK) st = init_state(b);
  if (st == BA_OK && cudaStreamSynchronize(h->s) != cudaSuccess) st = set_error(BA_ERR_CUDA, "batch set-up failed");
  if (st != BA_OK) {
    delete b;
    return st;
  }
  *out = b;
  return BA_OK;
}

ba_status ba_batch_destroy(ba_batch* b) {
  if (!b) return BA_OK;
  cudaStreamSynchronize(b->h->s);
  delete b;
  return BA_OK;
}

ba_status ba_batch_solve(ba_batch* b, int iters, void* stream) {
  if (!b) return set_error(BA_ERR_INVALID_ARG, "NULL batch");
  if (iters < 0) return set_error(BA_ERR_INVALID_ARG, "iters < 0");
  ba_status st = enter(b, stream);
  if (st != BA_OK) return st;
  st = enqueue_solve(b, iters);
  if (st != BA_OK) return st;
  return leave(b, stream);
}

ba_status ba_batch_get_params(ba_batch* b, void* cams_out, void* points_out, void* stream) {
  if (!b) return set_error(BA_ERR_INVALID_ARG, "NULL batch");
  ba_status st = enter(b, stream);
  if (st != BA_OK) return st;
  ba_problem* h = b->h;
  const long long n = std::max(h->C, h->P);
  if (h->prec == BA_PREC_F32)
    k_batch_params<float><<<nblk(n, 256), 256, 0, h->s>>>(b->nprob, h->C, h->P, b->d_cam_off, b->d_pt_off,
                                                          h->pnewpos, b->state, (const float*)h->cams,
                                                          (const float*)h->pts, (float*)cams_out, (float*)points_out);
  else
    k_batch_params<double><<<nblk(n, 256), 256, 0, h->s>>>(b->nprob, h->C, h->P, b->d_cam_off, b->d_pt_off,
                                                           h->pnewpos, b->state, (const double*)h->cams,
                                                           (const double*)h->pts, (double*)cams_out,
                                                           (double*)points_out);
  count_launch();
  BCU(cudaGetLastError());
  return leave(b, stream);
}

ba_status ba_batch_reset(ba_batch* b, const void* cams, const void* points, void* stream) {
  if (!b) return set_error(BA_ERR_INVALID_ARG, "NULL batch");
  ba_status st = enter(b, stream);
  if (st != BA_OK) return st;
  ba_problem* h = b->h;
  const size_t cb = 9ull * h->C * h->tsize, pb = 3ull * h->P * h->tsize;
  BCU(cudaMemcpyAsync(h->cams, cams ? cams : b->cams0, cb, cams ? cudaMemcpyDefault : cudaMemcpyDeviceToDevice, h->s));
  if (points) {
    // caller's point order -> internal order
    BCU(cudaMemcpyAsync(h->pts_tmp, points, pb, cudaMemcpyDefault, h->s));
    if (h->prec == BA_PREC_F32)
      k_gather_rows<float, 3><<<nblk(h->P, 256), 256, 0, h->s>>>(h->P, h->pnew, (const float*)h->pts_tmp,
                                                                 (float*)h->pts);
    else
      k_gather_rows<double, 3><<<nblk(h->P, 256), 256, 0, h->s>>>(h->P, h->pnew, (const double*)h->pts_tmp,
                                                                  (double*)h->pts);
    count_launch();
    BCU(cudaGetLastError());
  } else {
    BCU(cudaMemcpyAsync(h->pts, b->pts0, pb, cudaMemcpyDeviceToDevice, h->s));
  }
  st = init_state(b);
  if (st != BA_OK) return st;
  return leave(b, stream);
}

ba_status ba_batch_get_stats(ba_batch* b, ba_iter_stats* host_out, int cap, int* n_out) {
  if (!b || (cap > 0 && !host_out)) return set_error(BA_ERR_INVALID_ARG, "NULL argument");
  std::vector<BState> st(b->nprob);
  std::vector<ba_iter_stats> ring((size_t)b->nprob * b->cap);
  BCU(cudaMemcpyAsync(st.data(), b->state, st.size() * sizeof(BState), cudaMemcpyDeviceToHost, b->h->s));
  BCU(cudaMemcpyAsync(ring.data(), b->stats, ring.size() * sizeof(ba_iter_stats), cudaMemcpyDeviceToHost, b->h->s));
  BCU(cudaStreamSynchronize(b->h->s));
  int bad = 0;
  for (int i = 0; i < b->nprob; ++i) {
    const long long avail = std::min<long long>(st[i].trials, b->cap);
    const long long n = std::min<long long>(avail, cap > 0 ? cap : 0);
    for (long long k = 0; k < n; ++k) {
      const long long t = st[i].trials - n + k;
      host_out[(size_t)i * cap + k] = ring[(size_t)i * b->cap + t % b->cap];
    }
    if (n_out) n_out[i] = (int)n;
    bad += st[i].nonfinite;
    st[i].nonfinite = 0;
  }
  if (bad > 0) {
    BCU(cudaMemcpy(b->state, st.data(), st.size() * sizeof(BState), cudaMemcpyHostToDevice));
    return set_error(BA_ERR_NONFINITE, "%d trial(s) produced a non-finite cost and were rejected", bad);
  }
  return BA_OK;
}

ba_status ba_batch_get_scalars(ba_batch* b, double* cost, double* lambda) {
  if (!b) return set_error(BA_ERR_INVALID_ARG, "NULL batch");
  std::vector<BState> st(b->nprob);
  BCU(cudaMemcpyAsync(st.data(), b->state, st.size() * sizeof(BState), cudaMemcpyDeviceToHost, b->h->s));
  BCU(cudaStreamSynchronize(b->h->s));
  for (int i = 0; i < b->nprob; ++i) {
    if (cost) cost[i] = st[i].need_cost ? NAN : st[i].F;
    if (lambda) lambda[i] = st[i].lam;
  }
  return BA_OK;
}

ba_status ba_batch_set_launch(ba_batch* b, int ctas_per_sm, int variant, int order) {
  if (!b) return set_error(BA_ERR_INVALID_ARG, "NULL batch");
  if (ctas_per_sm < 1 || ctas_per_sm > 64 || (variant != 0 && variant != 1) || (order != 0 && order != 1))
    return set_error(BA_ERR_INVALID_ARG, "ctas_per_sm in [1, 64], variant and order in {0, 1}");
  BCU(cudaStreamSynchronize(b->h->s));
  b->ctas_per_sm = ctas_per_sm;
  b->variant = variant;
  if (order != b->order) {
    b->order = order;
    ba_status st = upload_order(b);
    if (st != BA_OK) return st;
  }
  return BA_OK;
}

ba_status ba_batch_set_segments(ba_batch* b, int piece_max, int chunk_slots, int chunk_pts) {
  if (!b) return set_error(BA_ERR_INVALID_ARG, "NULL batch");
  if (piece_max < 32 || piece_max > PIECE || chunk_slots < 32 || chunk_slots > CHUNK_SLOTS || chunk_pts < 1 ||
      chunk_pts > CHUNK_PTS)
    return set_error(BA_ERR_INVALID_ARG, "piece_max in [32, %d], chunk_slots in [32, %d], chunk_pts in [1, %d]",
                     PIECE, CHUNK_SLOTS, CHUNK_PTS);
  ba_problem* h = b->h;
  BCU(cudaStreamSynchronize(h->s));
  if (piece_max == b->piece_max && chunk_slots == b->chunk_slots && chunk_pts == b->chunk_pts) return BA_OK;
  const int C = h->C, P = h->P;
  std::vector<int32_t> rp(C + 1), rq(P + 1);
  BCU(cudaMemcpy(rp.data(), h->rowptr_cam, (C + 1) * 4ull, cudaMemcpyDeviceToHost));
  BCU(cudaMemcpy(rq.data(), h->rowptr_pt, (P + 1) * 4ull, cudaMemcpyDeviceToHost));
  // pieces: each camera's slots cut into equal runs of at most piece_max
  // (the single problem's cut with its maximum replaced)
  std::vector<int32_t> pc, pb, pe, cpp(C + 1);
  for (int c = 0; c < C; ++c) {
    cpp[c] = (int32_t)pc.size();
    const int n = rp[c + 1] - rp[c];
    const int k = (n + piece_max - 1) / piece_max;
    for (int i = 0; i < k; ++i) {
      pc.push_back(c);
      pb.push_back(rp[c] + (int)((long long)n * i / k));
      pe.push_back(rp[c] + (int)((long long)n * (i + 1) / k));
    }
  }
  cpp[C] = (int32_t)pc.size();
  if (pc.size() > b->piece_cap) {
    BCU(b->alloc(&h->piece_cam, pc.size() * 4));
    BCU(b->alloc(&h->piece_beg, pc.size() * 4));
    BCU(b->alloc(&h->piece_end, pc.size() * 4));
    BCU(b->alloc(&h->part, (size_t)PART * pc.size() * 8));
    b->piece_cap = pc.size();
  }
  BCU(cudaMemcpy(h->piece_cam, pc.data(), pc.size() * 4, cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(h->piece_beg, pb.data(), pb.size() * 4, cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(h->piece_end, pe.data(), pe.size() * 4, cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(h->cam_piece_ptr, cpp.data(), (C + 1) * 4ull, cudaMemcpyHostToDevice));
  h->npieces = (int)pc.size();
  std::vector<int32_t> bch = cut_chunks(b, rq, chunk_slots, chunk_pts);
  if (bch.size() > b->chunk_cap) {
    BCU(b->alloc(&b->d_bchunk, bch.size() * 4));
    BCU(b->alloc(&b->dot_gp, bch.size() * 8));
    b->chunk_cap = bch.size();
  }
  BCU(cudaMemcpy(b->d_bchunk, bch.data(), bch.size() * 4, cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(b->d_chunk_off, b->chunk_off.data(), (b->nprob + 1) * 4ull, cudaMemcpyHostToDevice));
  b->piece_max = piece_max;
  b->chunk_slots = chunk_slots;
  b->chunk_pts = chunk_pts;
  if (b->gexec) {  // the captured solve holds the old arrays
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  return BA_OK;
}

ba_status ba_batch_get_segments(ba_batch* b, int* piece_max, int* chunk_slots, int* chunk_pts) {
  if (!b) return set_error(BA_ERR_INVALID_ARG, "NULL batch");
  if (piece_max) *piece_max = b->piece_max;
  if (chunk_slots) *chunk_slots = b->chunk_slots;
  if (chunk_pts) *chunk_pts = b->chunk_pts;
  return BA_OK;
}

ba_status ba_batch_get_launch(ba_batch* b, int* ctas_per_sm, int* variant, int* order, int* grid) {
  if (!b) return set_error(BA_ERR_INVALID_ARG, "NULL batch");
  if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
  if (variant) *variant = b->variant;
  if (order) *order = b->order;
  if (grid) *grid = grid_of(b);
  return BA_OK;
}

ba_status ba_batch_autotune(ba_batch* b, int iters, const char* cache_path, double* best_ms) {
  if (!b || iters < 1) return set_error(BA_ERR_INVALID_ARG, "NULL batch or iters < 1");
  if (best_ms) *best_ms = 0.0;
  const std::string key = tune_key(b);
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string line, hit;
    const std::string pat = "\"key\": \"" + key + "\"";
    while (std::getline(in, line))
      if (line.find(pat) != std::string::npos) hit = line;  // the last entry wins
    int c = 0, v = 0, o = 0, pm = 0, cs = 0, cp = 0;
    if (!hit.empty() && json_int(hit, "ctas_per_sm", &c) && json_int(hit, "variant", &v) &&
        json_int(hit, "order", &o) && json_int(hit, "piece_max", &pm) && json_int(hit, "chunk_slots", &cs) &&
        json_int(hit, "chunk_pts", &cp) && ba_batch_set_segments(b, pm, cs, cp) == BA_OK &&
        ba_batch_set_launch(b, c, v, o) == BA_OK)
      return BA_OK;
  }
  ba_problem* h = b->h;
  const size_t cb = 2 * 9ull * h->C * h->tsize, pb = 2 * 3ull * h->P * h->tsize;
  const size_t sb = b->nprob * sizeof(BState), rb = (size_t)b->nprob * b->cap * sizeof(ba_iter_stats);
  // snapshot of everything a solve changes that outlives it
  void *sc = nullptr, *sp = nullptr, *ss = nullptr, *sr = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&sc, cb);
  if (e == cudaSuccess) e = cudaMalloc(&sp, pb);
  if (e == cudaSuccess) e = cudaMalloc(&ss, sb);
  if (e == cudaSuccess) e = cudaMalloc(&sr, rb);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sc, h->cams, cb, cudaMemcpyDeviceToDevice, h->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sp, h->pts, pb, cudaMemcpyDeviceToDevice, h->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ss, b->state, sb, cudaMemcpyDeviceToDevice, h->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sr, b->stats, rb, cudaMemcpyDeviceToDevice, h->s);
  auto restore = [&]() {
    cudaError_t r = cudaMemcpyAsync(h->cams, sc, cb, cudaMemcpyDeviceToDevice, h->s);
    if (r == cudaSuccess) r = cudaMemcpyAsync(h->pts, sp, pb, cudaMemcpyDeviceToDevice, h->s);
    if (r == cudaSuccess) r = cudaMemcpyAsync(b->state, ss, sb, cudaMemcpyDeviceToDevice, h->s);
    if (r == cudaSuccess) r = cudaMemcpyAsync(b->stats, sr, rb, cudaMemcpyDeviceToDevice, h->s);
    return r;
  };
  const int c0 = b->ctas_per_sm, v0 = b->variant, o0 = b->order;
  int bc = c0, bv = v0, bo = o0;
  float best = -1.f;
  ba_status st = BA_OK;
  for (int v = 0; v < 2 && e == cudaSuccess && st == BA_OK; ++v) {
    const int occ = std::min(occupancy(b, v), std::max(1, (b->nprob + b->nsm - 1) / b->nsm));
    for (int o = 0; o < 2 && e == cudaSuccess && st == BA_OK; ++o) {
      for (int c = 1; c <= occ && e == cudaSuccess && st == BA_OK; ++c) {
        st = ba_batch_set_launch(b, c, v, o);
        // warm-up (graph capture) then one timed solve, each from the snapshot
        for (int rep = 0; rep < 2 && st == BA_OK && e == cudaSuccess; ++rep) {
          e = restore();
          if (e == cudaSuccess && rep == 1) e = cudaEventRecord(e0, h->s);
          if (e == cudaSuccess) st = enqueue_solve(b, iters);
          if (e == cudaSuccess && st == BA_OK && rep == 1) e = cudaEventRecord(e1, h->s);
        }
        float ms = 0.f;
        if (e == cudaSuccess && st == BA_OK) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess && st == BA_OK) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && st == BA_OK && (best < 0.f || ms < best)) {
          best = ms;
          bc = c;
          bv = v;
          bo = o;
        }
      }
    }
  }
  // segment sizes at the chosen launch: pieces of at most 256..2048
  // camera-major slots, point chunks of 256 / 512 / 1024 slots.  Another cut
  // changes the summation order, so a candidate is kept only if every
  // problem's final cost is within 1e-6 (relative) of the current cut's.
  int bp = b->piece_max, bs = b->chunk_slots, bpt = b->chunk_pts;
  if (e == cudaSuccess && st == BA_OK) st = ba_batch_set_launch(b, bc, bv, bo);
  std::vector<BState> ref(b->nprob), got(b->nprob);
  auto timed_run = [&](float& ms, std::vector<BState>& fin) {
    for (int rep = 0; rep < 2 && st == BA_OK && e == cudaSuccess; ++rep) {
      e = restore();
      if (e == cudaSuccess && rep == 1) e = cudaEventRecord(e0, h->s);
      if (e == cudaSuccess) st = enqueue_solve(b, iters);
      if (e == cudaSuccess && st == BA_OK && rep == 1) e = cudaEventRecord(e1, h->s);
    }
    if (e == cudaSuccess && st == BA_OK) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess && st == BA_OK) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && st == BA_OK)
      e = cudaMemcpy(fin.data(), b->state, b->nprob * sizeof(BState), cudaMemcpyDeviceToHost);
  };
  float ref_ms = 0.f;
  if (e == cudaSuccess && st == BA_OK) timed_run(ref_ms, ref);
  if (e == cudaSuccess && st == BA_OK) best = std::min(best < 0.f ? ref_ms : best, ref_ms);
  const int pieces[] = {256, 512, 1024, PIECE};
  const int chunks[][2] = {{256, 128}, {512, 256}, {CHUNK_SLOTS, CHUNK_PTS}};
  const int p0 = bp, s0 = bs, t0 = bpt;
  float best_seg = ref_ms;
  for (int pm : pieces) {
    for (const auto& ck : chunks) {
      if (e != cudaSuccess || st != BA_OK) break;
      if (pm == p0 && ck[0] == s0 && ck[1] == t0) continue;
      st = ba_batch_set_segments(b, pm, ck[0], ck[1]);
      float ms = 0.f;
      if (st == BA_OK) timed_run(ms, got);
      if (e != cudaSuccess || st != BA_OK) break;
      bool same = true;
      for (int i = 0; i < b->nprob && same; ++i)
        same = std::isfinite(got[i].F) && std::fabs(got[i].F - ref[i].F) <= 1e-6 * std::fabs(ref[i].F);
      if (same && ms < best_seg) {
        best_seg = ms;
        bp = pm;
        bs = ck[0];
        bpt = ck[1];
      }
    }
  }
  if (e == cudaSuccess && st == BA_OK) {
    st = ba_batch_set_segments(b, bp, bs, bpt);
    best = best_seg;
  }
  if (e == cudaSuccess) e = restore();
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
  cudaFree(sc);
  cudaFree(sp);
  cudaFree(ss);
  cudaFree(sr);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st != BA_OK) return st;
  if (e != cudaSuccess) return set_error(BA_ERR_CUDA, "autotune failed: %s", cudaGetErrorString(e));
  st = ba_batch_set_launch(b, bc, bv, bo);
  if (st != BA_OK) return st;
  if (best_ms) *best_ms = best;
  if (cache_path) {
    FILE* f = fopen(cache_path, "a");
    if (f) {
      fprintf(f,
              "{\"key\": \"%s\", \"variant\": %d, \"ctas_per_sm\": %d, \"order\": %d, \"piece_max\": %d, "
              "\"chunk_slots\": %d, \"chunk_pts\": %d, \"ms\": %.4f, \"iters\": %d}\n",
              key.c_str(), bv, bc, bo, bp, bs, bpt, best, iters);
      fclose(f);
    }
  }
  return BA_OK;
}

}  // extern "C"
