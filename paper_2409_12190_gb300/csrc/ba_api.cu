// C ABI of the LM bundle-adjustment library (include/ba.h): the problem
// object, its device buffers, the stream-ordered LM trial and its CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "ba.h"
#include "ba_internal.h"
#include "ba_band.cuh"
#include "ba_kernels.cuh"
#include "ba_learn.cuh"
#include "ba_problem.h"

namespace ba {

static std::atomic<uint64_t> g_launches{0};
static thread_local bool g_capturing = false;

void count_launch(uint64_t n) {
  if (!g_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}

}  // namespace ba

namespace {

thread_local std::string g_err;

ba_status fail(ba_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CU(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      ba_status s_ = (e_ == cudaErrorMemoryAllocation) ? BA_ERR_OOM : BA_ERR_CUDA;      \
      return fail(s_, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                           \
    }                                                                                  \
  } while (0)

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

namespace ba {

ba_status set_error(ba_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

}  // namespace ba

namespace {

using namespace ba;

// Order the problem's internal stream after the caller's stream.
ba_status enter(ba_problem* h, void* stream) {
  CU(cudaEventRecord(h->ev_in, (cudaStream_t)stream));
  CU(cudaStreamWaitEvent(h->s, h->ev_in, 0));
  return BA_OK;
}
// Order the caller's stream after the problem's internal stream.
ba_status leave(ba_problem* h, void* stream) {
  CU(cudaEventRecord(h->ev_out, h->s));
  CU(cudaStreamWaitEvent((cudaStream_t)stream, h->ev_out, 0));
  return BA_OK;
}

// Event pair around one launch when profiling is on (no-op otherwise).
struct Prof {
  ba_problem* h;
  ba_problem::ProfRec rec{};
  Prof(ba_problem* hh, int kind, int k = -1) : h(hh) {
    if (!h->prof) return;
    rec.kind = kind;
    rec.trial = h->prof_trial;
    rec.k = k;
    cudaEventCreate(&rec.a);
    cudaEventCreate(&rec.b);
    cudaEventRecord(rec.a, h->s);
  }
  ~Prof() {
    if (!h->prof) return;
    cudaEventRecord(rec.b, h->s);
    h->prof->push_back(rec);
  }
};

// One exchange of a point-partitioned problem: buf[0 .. n) <- its sum over
// every part (the caller's all-reduce on the problem's stream).  The first
// failure is kept in h->xerr and reported after the trial.
void xchg(ba_problem* h, double* buf, size_t n) {
  if (h->xerr) return;
  if (n > h->xcap || cudaMemcpyAsync(h->xbuf, buf, n * 8, cudaMemcpyDeviceToDevice, h->s) != cudaSuccess) {
    h->xerr = 1;
    return;
  }
  if (h->xch(n, (void*)h->s, h->xctx) != 0) {
    h->xerr = 2;
    return;
  }
  if (cudaMemcpyAsync(buf, h->xbuf, n * 8, cudaMemcpyDeviceToDevice, h->s) != cudaSuccess) h->xerr = 1;
}

template <typename T, bool MF>
void enqueue_lin(ba_problem* h, int gate) {
  cudaStream_t s = h->s;
  const T delta = (T)(h->opt.huber_delta > 0 ? h->opt.huber_delta : 0.0);
  {
    Prof pr(h, BA_K_OTHER, -2);
    k_cam_prep<T><<<nblk(h->C, 128), 128, 0, s>>>(h->C, (const T*)h->cams, h->st, gate, (T*)h->camtab);
  }
  {
    Prof pr(h, BA_K_OTHER, -2);
    k_pt_prep<T><<<nblk(h->P, 256), 256, 0, s>>>(h->P, (const T*)h->pts, h->st, gate, (T*)h->ptab);
  }
  {
    Prof pr(h, BA_K_LIN_CAM, -2);
    k_lin_cam<T, !MF><<<h->npieces, LIN_THREADS, 0, s>>>(
        h->piece_cam, h->piece_beg, h->piece_end, h->cm_pt, (const T*)h->cm_px, (const T*)h->pts,
        (const T*)h->camtab, h->st, gate, delta, h->O, h->P, (T*)h->Jcm, (T*)h->cm_sw, h->part);
  }
  {
    Prof pr(h, BA_K_OTHER, -2);
    k_cam_combine_lin<<<nblk(h->C, 128), 128, 0, s>>>(h->C, h->cam_piece_ptr, h->part, h->st, gate,
                                                      h->xch ? h->U_loc : h->U, h->xch ? h->gc_loc : h->gc);
  }
  if (h->xch) {
    // U and gc over every part (this part's, kept, summed again each trial:
    // a skipped linearisation leaves the same sums)
    cudaMemcpyAsync(h->U, h->U_loc, 45ull * h->C * 8, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(h->gc, h->gc_loc, 9ull * h->C * 8, cudaMemcpyDeviceToDevice, s);
    xchg(h, h->U, 45ull * h->C);
    xchg(h, h->gc, 9ull * h->C);
  }
  if (!MF && h->Jpm) {
    Prof pr(h, BA_K_OTHER, -2);
    k_planes_pm<T><<<nblk(h->O, 256), 256, 0, s>>>(h->O, h->st, gate, h->pm2cm, (const T*)h->Jcm, (T*)h->Jpm);
    count_launch();
  }
  {
    Prof pr(h, BA_K_LIN_PT, -2);
    k_lin_pt<T><<<h->nchunks, CHUNK_THREADS, lin_pt_smem<T>(h->fa), s>>>(
        h->pchunk, h->O, h->rowptr_pt, h->pm_cam, h->pm_pt, (const T*)h->pm_px, (const T*)h->pts,
        (const T*)h->camtab, h->st, h->P, gate, delta, (T*)h->pm_sw, h->V, h->gp, h->fa ? h->chunk_hdr : nullptr,
        h->pm_lc, h->chunk_cams);
  }
  count_launch(5);
}

// Passes A1, A2 (MODE 0) and B of S p for p in the pass form xc: t in the
// point table, pass-B partials in h->part.  k = PCG iteration (profiling).
template <typename T, bool MF>
void enqueue_schur_product(ba_problem* h, const T* xc, int k, int check_done) {
  cudaStream_t s = h->s;
  if (MF && h->fa) {
    {
      Prof pr(h, BA_K_PASS_FA, k);
      auto fa = h->pm_sw ? k_pass_fa<T, 0, true> : k_pass_fa<T, 0, false>;
      fa<<<h->nchunks, CHUNK_THREADS, fa_smem<T>(h->fa_nc), s>>>(
          h->pchunk, h->P, h->rowptr_pt, h->pm_pt, h->pm_lc, (const T*)h->pm_sw, h->chunk_cams, h->chunk_cam_ptr,
          (const T*)h->camtab, xc, (const T*)h->Vinv, h->st, check_done, (T*)h->ptab, nullptr, nullptr, nullptr,
          nullptr, nullptr, h->chunk_hdr, h->fa_nc);
    }
    {
      Prof pr(h, BA_K_PASS_B, k);
      // FP32 recompute mode: two gathers in flight per thread, next indices prefetched
      constexpr int UB = (MF && std::is_same<T, float>::value) ? 2 : 1;
      constexpr int NT = UB > 1 ? PASSB_THREADS : PIECE_THREADS;
      auto pb = h->cm_sw ? k_pass_b<T, MF, UB, (UB > 1), NT, true> : k_pass_b<T, MF, UB, (UB > 1), NT, false>;
      pb<<<h->npieces, NT, 0, s>>>(
          h->piece_cam, h->piece_beg, h->piece_end, h->cm_pt, (const T*)h->Jcm, (const T*)h->cm_sw,
          (const T*)h->ptab, (const T*)h->camtab, h->st, check_done, h->O, h->part);
    }
    count_launch(2);
    return;
  }
  if (!MF && h->Jpm) {
    {
      Prof pr(h, BA_K_PASS_FA, k);
      k_pass_fs<T><<<h->nchunks, CHUNK_THREADS, fs_smem<T>(h->fa_nc), s>>>(
          h->rowptr_pt, h->pm_lc, h->chunk_cams, (const T*)h->Jpm, h->O, xc, (const T*)h->Vinv, h->st,
          check_done, (T*)h->ptab, h->chunk_hdr, h->fa_nc);
    }
    {
      Prof pr(h, BA_K_PASS_B, k);
      k_pass_b<T, MF><<<h->npieces, PIECE_THREADS, 0, s>>>(
          h->piece_cam, h->piece_beg, h->piece_end, h->cm_pt, (const T*)h->Jcm, (const T*)h->cm_sw,
          (const T*)h->ptab, (const T*)h->camtab, h->st, check_done, h->O, h->part);
    }
    count_launch(2);
    return;
  }
  {
    Prof pr(h, BA_K_PASS_A, k);
    k_pass_a1<T, MF><<<h->npieces, PIECE_THREADS, 0, s>>>(
        h->piece_cam, h->piece_beg, h->piece_end, h->cm_pt, (const T*)h->Jcm, (const T*)h->cm_sw,
        (const T*)h->ptab, (const T*)h->camtab, xc, h->st, check_done, h->O, (T*)h->zbuf);
  }
  {
    Prof pr(h, BA_K_PASS_A2, k);
    k_pass_a2<T, 0><<<h->nchunks, CHUNK_THREADS, CHUNK_SLOTS * 4 * sizeof(T), s>>>(
        h->pchunk, h->P, h->rowptr_pt, h->pm2cm, (const T*)h->zbuf, (const T*)h->Vinv, h->st, check_done,
        (T*)h->ptab, nullptr, nullptr, nullptr, nullptr, nullptr);
  }
  {
    Prof pr(h, BA_K_PASS_B, k);
    constexpr int UB = (MF && std::is_same<T, float>::value) ? 2 : 1;
    constexpr int NT = UB > 1 ? PASSB_THREADS : PIECE_THREADS;
    auto pb = h->cm_sw ? k_pass_b<T, MF, UB, (UB > 1), NT, true> : k_pass_b<T, MF, UB, (UB > 1), NT, false>;
    pb<<<h->npieces, NT, 0, s>>>(
        h->piece_cam, h->piece_beg, h->piece_end, h->cm_pt, (const T*)h->Jcm, (const T*)h->cm_sw,
        (const T*)h->ptab, (const T*)h->camtab, h->st, check_done, h->O, h->part);
  }
  count_launch(3);
}

// One PCG pass pair plus the vector updates of iteration k.
template <typename T, bool MF>
void enqueue_pcg_iter(ba_problem* h, const double* lam_ptr, int k, double tol) {
  cudaStream_t s = h->s;
  const double dmin = h->opt.diag_min, dmax = h->opt.diag_max;
  enqueue_schur_product<T, MF>(h, (const T*)h->pT, k, 1);
  if (h->xch) {
    // the pass-B sums of every part (9C values), one row per camera
    k_cam_sum_parts<<<nblk(9LL * h->C, 256), 256, 0, s>>>(h->C, h->cam_piece_ptr, h->part, 9, 9, h->camsum);
    count_launch();
    xchg(h, h->camsum, 9ull * h->C);
    Prof pr(h, BA_K_OTHER, k);
    k_pcg_q<T, MF, 9><<<h->ncb, VT, 0, s>>>(h->C, h->ident_ptr, h->camsum, h->U, (const T*)h->camtab, lam_ptr,
                                           dmin, dmax, h->p, h->q, h->dot_pq, h->fixed, h->st, 1);
  } else {
    Prof pr(h, BA_K_OTHER, k);
    k_pcg_q<T, MF><<<h->ncb, VT, 0, s>>>(h->C, h->cam_piece_ptr, h->part, h->U, (const T*)h->camtab, lam_ptr,
                                        dmin, dmax, h->p, h->q, h->dot_pq, h->fixed, h->st, 1);
  }
  count_launch(3);
  {
    Prof pr(h, BA_K_OTHER, k);
    k_pcg_update<<<h->ncb, VT, 0, s>>>(h->C, h->ncb, k, h->dot_pq, h->dot_rz, h->dot_rr, h->p, h->q, h->x, h->r,
                                       h->z, h->Minv, h->st);
  }
  {
    Prof pr(h, BA_K_OTHER, k);
    k_pcg_direction<T, MF><<<h->ncb, VT, 0, s>>>(h->C, h->ncb, k, tol, h->dot_rz, h->dot_rr,
                                                         h->dot_bb, h->z, h->p, (const T*)h->camtab, (T*)h->pT,
                                                         h->st);
  }
  count_launch(2);
}

// The learned correction's coupling feature: COUPLING_PROBES implicit
// Schur products with the SplitMix64 probes, summed per camera into h->kap
// (needs h->Sii; uses the PCG's p, pT and q, which the PCG start rewrites).
template <typename T, bool MF>
void enqueue_coupling(ba_problem* h, const double* lam_ptr) {
  cudaStream_t s = h->s;
  const double dmin = h->opt.diag_min, dmax = h->opt.diag_max;
  for (int k = 0; k < COUPLING_PROBES; ++k) {
    k_coup_probe_in<T, MF><<<nblk(h->C, 128), 128, 0, s>>>(h->C, k, h->Sii, (const T*)h->camtab, h->p, (T*)h->pT);
    enqueue_schur_product<T, MF>(h, (const T*)h->pT, -1, 0);
    k_pcg_q<T, MF><<<h->ncb, VT, 0, s>>>(h->C, h->cam_piece_ptr, h->part, h->U, (const T*)h->camtab, lam_ptr,
                                        dmin, dmax, h->p, h->q, nullptr, h->fixed, h->st, 0);
    k_coup_acc<<<nblk(h->C, 128), 128, 0, s>>>(h->C, k, h->Sii, h->q, h->kap);
    count_launch(3);
  }
}

// The direct solve of the reduced system (BA_SOLVER_CHOLESKY): explicit S in
// nseg partials, summed into the band tiles, then the factorisation and both
// triangular solves in one cooperative launch (ba_band.cuh); dc into h->x as
// the PCG would leave it.
template <typename T, bool MF>
void enqueue_dense_solve(ba_problem* h, const double* lam_ptr) {
  cudaStream_t s = h->s;
  const int n = 9 * h->C;
  Prof pr(h, BA_K_OTHER);
  k_dense_w<T, MF><<<nblk(h->P, DENSE_THREADS), DENSE_THREADS, 0, s>>>(
      h->P, h->rowptr_pt, h->pm_cam, h->pm2cm, (const T*)h->Jcm, (const T*)h->cm_sw, (const T*)h->camtab,
      (const T*)h->pts, h->st, h->O, h->Wd);
  k_schur_dense<T><<<h->C * h->nseg, DENSE_THREADS, 0, s>>>(
      h->C, h->nseg, h->rowptr_cam, h->cm_pt, h->rowptr_pt, h->pm_cam, h->pm2cm, h->Wd, (const T*)h->Vinv, h->Spart);
  count_launch();
  cudaMemsetAsync(h->bT, 0, h->bT_bytes, s);
  cudaMemsetAsync(h->bflag, 0, sizeof(int) * h->bflag_count, s);
  k_schur_to_band<<<n, 256, 0, s>>>(h->C, h->nseg, h->Spart, h->U, lam_ptr, h->opt.diag_min, h->opt.diag_max,
                                    h->fixed, h->bwt, h->bT);
  count_launch(2);
  if (h->bnb * BAND_TB > n) {
    k_band_pad<<<1, BAND_TB, 0, s>>>(n, h->bnb, h->bwt, h->bT);
    count_launch();
  }
  const size_t ntile = (size_t)h->bnb * (h->bwt + 1);
  int* ctr = h->bflag + 2 * ntile;
  BandArgs ba_{h->bnb, h->bwt, n, h->bntask, h->bncrit, h->band_crit, h->btask, h->bT, h->brs, h->bUi, h->r,
               h->dy, h->x, h->bflag, h->bflag + ntile, ctr, ctr + 5, ctr + 6};
  void* args[] = {&ba_};
  cudaLaunchCooperativeKernel((const void*)k_band_chol, dim3(h->band_grid), dim3(BAND_THREADS), args, 0, s);
  k_band_finish<<<nblk(n, 256), 256, 0, s>>>(n, ctr + 5, ctr, h->x, h->st);
  count_launch(2);
}

template <typename T, bool MF>
// chunk > 0 (direct launches only: not under capture, not a partitioned
// problem): enqueue the PCG iterations chunk at a time and stop once the
// device reports convergence, instead of enqueueing all maxiter of them
// (the iterations after convergence return at once, but each is still
// several launches).
void enqueue_solve(ba_problem* h, const double* lam_ptr, int maxiter, double tol, bool learned = false,
                   int chunk = 0) {
  cudaStream_t s = h->s;
  const double dmin = h->opt.diag_min, dmax = h->opt.diag_max;
  {
    Prof pr(h, BA_K_OTHER);
    k_pt_damp<T><<<nblk(h->P, PT_THREADS), PT_THREADS, 0, s>>>(h->P, h->V, h->gp, lam_ptr, dmin, dmax,
                                                              (T*)h->Vinv, (T*)h->y0);
  }
  {
    Prof pr(h, BA_K_SCHUR_CAM);
    k_schur_cam<T, MF><<<h->npieces, LIN_THREADS, 0, s>>>(
        h->piece_cam, h->piece_beg, h->piece_end, h->cm_pt, (const T*)h->Jcm, (const T*)h->camtab,
        (const T*)h->pts, (const T*)h->cm_sw, h->st, h->P, (const T*)h->Vinv, (const T*)h->y0, h->O, h->part);
  }
  const int32_t* sptr = h->cam_piece_ptr;
  const double* spart = h->part;
  if (h->xch) {
    // the per-camera Schur sums over every part, one row per camera
    k_cam_sum_parts<<<nblk(54LL * h->C, 256), 256, 0, s>>>(h->C, h->cam_piece_ptr, h->part, 54, PART, h->camsum);
    count_launch();
    xchg(h, h->camsum, (size_t)PART * h->C);
    sptr = h->ident_ptr;
    spart = h->camsum;
  }
  {
    Prof pr(h, BA_K_OTHER);
    k_cam_combine_schur<T, MF><<<h->ncb, CAM_THREADS, 0, s>>>(
        h->C, sptr, spart, h->U, h->gc, (const T*)h->camtab, lam_ptr, dmin, dmax, h->Minv, h->x,
        h->r, h->z, h->p, (T*)h->pT, h->dot_rz + h->ncb, h->dot_bb, h->fixed, h->st, learned ? h->Sii : nullptr);
  }
  count_launch(3);
  if (learned) {
    // the learned correction of the block-Jacobi blocks: features, network
    // (tensor cores), SPD blocks and the PCG start with them
    Prof pr(h, BA_K_OTHER);
    enqueue_coupling<T, MF>(h, lam_ptr);
    k_learn_features<<<h->ncb, CAM_THREADS, 0, s>>>(h->C, h->Sii, h->U, lam_ptr, dmin, dmax, h->rowptr_cam, h->Xf,
                                                    nullptr, nullptr, h->kap);
    k_mlp_forward<<<nblk(h->C, MLP_ROWS), MLP_THREADS, MLP_SMEM_FWD, s>>>(h->C, h->mlp, h->Xf, h->Ef);
    k_learn_start<T, MF><<<h->ncb, CAM_THREADS, 0, s>>>(h->C, h->Sii, h->Ef, (const T*)h->camtab, h->Minv, h->r,
                                                         h->z, h->p, (T*)h->pT, h->dot_rz + h->ncb, h->fixed,
                                                         h->st);
    count_launch(3);
  }
  if (h->opt.solver == BA_SOLVER_CHOLESKY) {
    enqueue_dense_solve<T, MF>(h, lam_ptr);
  } else {
    for (int k = 0; k < maxiter; ++k) {
      enqueue_pcg_iter<T, MF>(h, lam_ptr, k, tol);
      if (chunk > 0 && !h->xch && (k + 1) % chunk == 0 && k + 1 < maxiter) {
        int done = 0;
        if (cudaMemcpyAsync(&done, &h->st->pcg_done, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            cudaStreamSynchronize(s) == cudaSuccess && done)
          break;
      }
    }
  }
  {
    Prof pr(h, BA_K_OTHER);
    k_cam_trial<T, MF><<<h->ncb, CAM_THREADS, 0, s>>>(h->C, h->x, h->gc, (T*)h->cams, (const T*)h->camtab, h->st,
                                                     (T*)h->xT, h->dot_gc);
  }
  if (MF && h->fa) {
    Prof pr(h, BA_K_BACKSUB);
    auto fa = h->pm_sw ? k_pass_fa<T, 1, true> : k_pass_fa<T, 1, false>;
    fa<<<h->nchunks, CHUNK_THREADS, fa_smem<T>(h->fa_nc), s>>>(
        h->pchunk, h->P, h->rowptr_pt, h->pm_pt, h->pm_lc, (const T*)h->pm_sw, h->chunk_cams, h->chunk_cam_ptr,
        (const T*)h->camtab, (const T*)h->xT, (const T*)h->Vinv, h->st, 0, (T*)h->ptab, (T*)h->dp, (const T*)h->y0,
        h->gp, (T*)h->pts, h->dot_gp, h->chunk_hdr, h->fa_nc);
    count_launch(2);
    return;
  }
  {
    Prof pr(h, BA_K_BACKSUB);
    k_pass_a1<T, MF><<<h->npieces, PIECE_THREADS, 0, s>>>(
        h->piece_cam, h->piece_beg, h->piece_end, h->cm_pt, (const T*)h->Jcm, (const T*)h->cm_sw,
        (const T*)h->ptab, (const T*)h->camtab, (const T*)h->xT, h->st, 0, h->O, (T*)h->zbuf);
  }
  {
    Prof pr(h, BA_K_BACKSUB);
    k_pass_a2<T, 1><<<h->nchunks, CHUNK_THREADS, CHUNK_SLOTS * 4 * sizeof(T), s>>>(
        h->pchunk, h->P, h->rowptr_pt, h->pm2cm, (const T*)h->zbuf, (const T*)h->Vinv, h->st, 0, (T*)h->ptab,
        (T*)h->dp, (const T*)h->y0, h->gp, (T*)h->pts, h->dot_gp);
  }
  count_launch(3);
}

// F at theta into the device state; gated: only if marked stale.
template <typename T, bool MF>
void enqueue_cost(ba_problem* h, bool gated = false) {
  const T delta = (T)(h->opt.huber_delta > 0 ? h->opt.huber_delta : 0.0);
  k_cost_cam<T, false, MF><<<h->npieces, PIECE_THREADS, 0, h->s>>>(
      h->piece_cam, h->piece_beg, h->piece_end, h->cm_pt, (const T*)h->cm_px, (const T*)h->cams,
      (const T*)h->pts, h->st, gated ? 2 : 0, delta, h->C, h->P, h->O, nullptr, nullptr, nullptr, nullptr, nullptr,
      h->part);
  if (h->xch) {
    // the cost over every part (0 from each part when F is not stale)
    k_part_cost_sum<<<1, 256, 0, h->s>>>(h->npieces, h->part, h->st, gated ? 1 : 0, h->xscal + 4);
    xchg(h, h->xscal + 4, 1);
    k_cost_set<<<1, 1, 0, h->s>>>(h->st, gated ? 1 : 0, h->xscal + 4);
    count_launch(3);
    return;
  }
  k_cost_finalize<<<1, 256, 0, h->s>>>(h->npieces, h->part, h->st, gated ? 1 : 0);
  count_launch(2);
}

template <typename T, bool MF>
void enqueue_trial(ba_problem* h) {
  enqueue_cost<T, MF>(h, true);  // F if the parameters or pixels were replaced
  enqueue_lin<T, MF>(h, 1);
  enqueue_solve<T, MF>(h, &h->st->lam, h->opt.pcg_maxiter, h->opt.pcg_tol, h->learned);
  const T delta = (T)(h->opt.huber_delta > 0 ? h->opt.huber_delta : 0.0);
  {
    Prof pr(h, BA_K_COST);
    // FP32 recompute mode: 16 slots per thread, as in pass B
    constexpr int NT = (MF && std::is_same<T, float>::value) ? PASSB_THREADS : PIECE_THREADS;
    k_cost_cam<T, true, MF, NT><<<h->npieces, NT, 0, h->s>>>(
        h->piece_cam, h->piece_beg, h->piece_end, h->cm_pt, (const T*)h->cm_px, (const T*)h->cams,
        (const T*)h->pts, h->st, 1, delta, h->C, h->P, h->O, (const T*)h->Jcm, (const T*)h->cm_sw,
        (const T*)h->camtab, (const T*)h->xT, (const T*)h->dp, h->part);
  }
  const ba_options& o = h->opt;
  {
    Prof pr(h, BA_K_OTHER);
    // one block sums the per-piece and per-chunk partials (a few thousand
    // strided doubles): 1024 threads keep more of those loads in flight
    if (h->xch) {
      k_part_trial_sums<<<1, 1024, 0, h->s>>>(h->npieces, h->part, h->nchunks, h->dot_gp, h->xscal);
      count_launch();
      xchg(h, h->xscal, 3);
    }
    k_lm_control<<<1, 1024, 0, h->s>>>(h->npieces, h->part, h->ncb, h->dot_gc, h->nchunks, h->dot_gp, o.up, o.down,
                                      o.rho_good, o.rho_bad, o.lambda_min, o.lambda_max, h->st, h->stats, h->cap,
                                      h->xch ? h->xscal : nullptr);
  }
  count_launch(2);
}


// Call FN<T, MF>(h, args...) for the problem's precision and Jacobian mode.
#define BA_DISPATCH(h, FN, ...)                        \
  do {                                                 \
    if ((h)->prec == BA_PREC_F32) {                    \
      if ((h)->mf) FN<float, true>(h, ##__VA_ARGS__);  \
      else FN<float, false>(h, ##__VA_ARGS__);         \
    } else {                                           \
      if ((h)->mf) FN<double, true>(h, ##__VA_ARGS__); \
      else FN<double, false>(h, ##__VA_ARGS__);        \
    }                                                  \
  } while (0)

void enqueue_trial_any(ba_problem* h) { BA_DISPATCH(h, enqueue_trial); }

// Implicit-function adjoint at the current parameters: v = H*^{-1} dL/dtheta
// through the forward Schur/PCG solver (its gradient slots hold -dL/dtheta),
// then dL/dx_k = w_k J_k v and dL/dtheta0 on frozen parameters.
template <typename T, bool MF>
void enqueue_backward(ba_problem* h, const double* lam_ptr, int maxiter, double tol, const void* dLc,
                      const void* dLp, void* dpix, void* dc0, void* dp0) {
  cudaStream_t s = h->s;
  enqueue_lin<T, MF>(h, 1);
  const long long n = std::max(9LL * h->C, 3LL * h->P);
  k_adj_rhs<T><<<nblk(n, 256), 256, 0, s>>>(h->C, h->P, (const T*)dLc, (const T*)dLp, h->pnew, h->gc, h->gp);
  count_launch();
  enqueue_solve<T, MF>(h, lam_ptr, maxiter, tol, false, 16);
  const T delta = (T)(h->opt.huber_delta > 0 ? h->opt.huber_delta : 0.0);
  k_adjoint_cam<T, MF><<<h->npieces, PIECE_THREADS, 0, s>>>(
      h->piece_cam, h->piece_beg, h->piece_end, h->cm_pt, h->perm_cam, (const T*)h->cm_px, (const T*)h->Jcm,
      (const T*)h->cm_sw, (const T*)h->ptab, (const T*)h->camtab, (const T*)h->xT, (const T*)h->dp, delta, h->O,
      (T*)dpix, h->part);
  count_launch();
  if (dc0) {
    k_adjoint_combine<T, MF><<<nblk(h->C, 128), 128, 0, s>>>(h->C, h->cam_piece_ptr, h->part, h->U,
                                                            (const T*)h->camtab, lam_ptr, h->opt.diag_min,
                                                            h->opt.diag_max, h->x, (const T*)dLc, h->fixed, (T*)dc0);
    count_launch();
  }
}

template <typename T, bool MF>
void launch_export(ba_problem* h, void* Jc, void* Jp, void* w) {
  const T delta = (T)(h->opt.huber_delta > 0 ? h->opt.huber_delta : 0.0);
  k_export_lin<T, MF><<<nblk(h->O, 256), 256, 0, h->s>>>(
      h->O, h->P, h->perm_cam, h->cam_idx, h->cm_pt, (const T*)h->cm_px, (const T*)h->Jcm, (const T*)h->cm_sw,
      (const T*)h->camtab, (const T*)h->pts, h->st, delta, (T*)Jc, (T*)Jp, (T*)w);
  count_launch();
}

// q = S p for p already in h->p (double), damped with *lam_ptr; no PCG state.
template <typename T, bool MF>
void enqueue_matvec(ba_problem* h, const double* lam_ptr) {
  cudaStream_t s = h->s;
  const double dmin = h->opt.diag_min, dmax = h->opt.diag_max;
  k_pt_damp<T><<<nblk(h->P, PT_THREADS), PT_THREADS, 0, s>>>(h->P, h->V, h->gp, lam_ptr, dmin, dmax, (T*)h->Vinv,
                                                            (T*)h->y0);
  k_pass_vec<T, MF><<<nblk(h->C, 128), 128, 0, s>>>(h->C, h->p, (const T*)h->camtab, (T*)h->pT);
  enqueue_schur_product<T, MF>(h, (const T*)h->pT, -1, 0);
  k_pcg_q<T, MF><<<h->ncb, VT, 0, s>>>(h->C, h->cam_piece_ptr, h->part, h->U, (const T*)h->camtab, lam_ptr,
                                      dmin, dmax, h->p, h->q, nullptr, h->fixed, h->st, 0);
  count_launch(3);
}

ba_status check_options(const ba_options* o) {
  if (o->precision != BA_PREC_F64 && o->precision != BA_PREC_F32)
    return fail(BA_ERR_INVALID_ARG, "precision must be BA_PREC_F64 or BA_PREC_F32");
  if (!(o->lambda0 > 0) || !(o->up > 1) || !(o->down > 0 && o->down < 1) || !(o->lambda_min > 0) ||
      !(o->lambda_max >= o->lambda_min) || !(o->diag_min >= 0) || !(o->diag_max >= o->diag_min))
    return fail(BA_ERR_INVALID_ARG, "damping options out of range");
  if (o->pcg_maxiter < 0 || o->pcg_maxiter > 100000 || !(o->pcg_tol >= 0))
    return fail(BA_ERR_INVALID_ARG, "pcg_maxiter must be in [0, 100000] and pcg_tol >= 0");
  if (o->max_stats < 1 || o->max_stats > (1 << 24)) return fail(BA_ERR_INVALID_ARG, "max_stats out of range");
  if (!(o->huber_delta >= 0) && !(o->huber_delta <= 0))
    return fail(BA_ERR_INVALID_ARG, "huber_delta is NaN");
  if (o->jacobian_mode < BA_JAC_AUTO || o->jacobian_mode > BA_JAC_STORE)
    return fail(BA_ERR_INVALID_ARG, "jacobian_mode must be BA_JAC_AUTO, BA_JAC_RECOMPUTE or BA_JAC_STORE");
  if (o->solver != BA_SOLVER_PCG && o->solver != BA_SOLVER_CHOLESKY)
    return fail(BA_ERR_INVALID_ARG, "solver must be BA_SOLVER_PCG or BA_SOLVER_CHOLESKY");
  return BA_OK;
}

template <typename T>
ba_status create_impl(ba_problem* h, const void* cams, const void* points, const int32_t* cam_idx,
                      const int32_t* pt_idx, const void* pixels) {
  const long long C = h->C, P = h->P, O = h->O;
  const size_t ts = sizeof(T);
  cudaStream_t s = h->s;
  CU(h->alloc(&h->st, sizeof(DevState)));
  CU(cudaMemsetAsync(h->st, 0, sizeof(DevState), s));
  {
    DevState init{};
    init.lam = h->opt.lambda0;
    init.lam_probe = h->opt.lambda0;
    init.need_lin = 1;
    CU(cudaMemcpyAsync(h->st, &init, sizeof(DevState), cudaMemcpyHostToDevice, s));
  }
  CU(h->alloc(&h->cams, 2 * 9 * C * ts));
  CU(h->alloc(&h->pts, 2 * 3 * P * ts));
  CU(h->alloc(&h->cam_idx, O * 4));
  CU(h->alloc(&h->pt_idx, O * 4));
  CU(h->alloc(&h->px_in, 2 * O * ts));
  CU(cudaMemcpyAsync(h->cams, cams, 9 * C * ts, cudaMemcpyDefault, s));
  CU(cudaMemcpyAsync(h->pts, points, 3 * P * ts, cudaMemcpyDefault, s));
  CU(cudaMemcpyAsync(h->cam_idx, cam_idx, O * 4, cudaMemcpyDefault, s));
  CU(cudaMemcpyAsync(h->pt_idx, pt_idx, O * 4, cudaMemcpyDefault, s));
  CU(cudaMemcpyAsync(h->px_in, pixels, 2 * O * ts, cudaMemcpyDefault, s));
  const long long nv = std::max(O, std::max(9 * C, 3 * P));
  k_validate<T><<<nblk(nv, 256), 256, 0, s>>>(h->C, h->P, h->O, (const T*)h->cams, (const T*)h->pts,
                                              h->cam_idx, h->pt_idx, (const T*)h->px_in, h->st);
  count_launch();
  int err = 0;
  CU(cudaMemcpyAsync(&err, &h->st->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (err & 1) return fail(BA_ERR_INVALID_ARG, "observation index out of range");
  if (err & 2) return fail(BA_ERR_NONFINITE, "non-finite camera, point or pixel value");

  // symbolic phase (Sec. IV-B), in the caller's numbering: stable sorts of the
  // observations by camera and by point
  CU(h->alloc(&h->xperm_cam, O * 4));
  CU(h->alloc(&h->xperm_pt, O * 4));
  CU(h->alloc(&h->rowptr_cam, (C + 1) * 4));
  CU(h->alloc(&h->xrowptr_pt, (P + 1) * 4));
  CU(h->alloc(&h->perm_cam, O * 4));
  CU(h->alloc(&h->perm_pt, O * 4));
  CU(h->alloc(&h->rowptr_pt, (P + 1) * 4));
  CU(h->alloc(&h->pnew, P * 4));
  CU(h->alloc(&h->pnewpos, P * 4));
  CU(h->alloc(&h->pts_tmp, 3 * P * ts));
  CU(h->alloc(&h->cams_tmp, 9 * C * ts));
  {
    const long long nmax = std::max(O, P);
    void* scratch = nullptr;
    int32_t *key = nullptr, *tmp = nullptr, *ptx = nullptr;
    CU(cudaMalloc(&scratch, csr_scratch_bytes((int)nmax)));
    cudaError_t e = cudaMalloc(&key, std::max(O, P + C + 2) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, std::max(O, P + 1) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&ptx, std::max(O, C + 1) * 4);
    int* derr = &h->st->err;
    if (e == cudaSuccess) e = csr_build_async(h->cam_idx, h->O, h->C, h->xperm_cam, h->rowptr_cam, scratch, derr, s);
    if (e == cudaSuccess) e = csr_build_async(h->pt_idx, h->O, h->P, h->xperm_pt, h->xrowptr_pt, scratch, derr, s);
    // renumber the points by the first camera that observes them (stable)
    if (e == cudaSuccess) {
      k_point_key<<<nblk(P, 256), 256, 0, s>>>(h->P, h->C, h->xrowptr_pt, h->xperm_pt, h->cam_idx, key);
      e = csr_build_async(key, h->P, h->C + 1, h->pnew, key + P, scratch, derr, s);
    }
    if (e == cudaSuccess) {
      k_invert_perm<<<nblk(P, 256), 256, 0, s>>>(h->P, h->pnew, h->pnewpos);
      k_gather_i32<<<nblk(O, 256), 256, 0, s>>>(h->O, h->pt_idx, h->pnewpos, ptx);  // internal point index
      e = cudaMemcpyAsync(h->pts_tmp, h->pts, 3 * P * ts, cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess) {
      k_gather_rows<T, 3><<<nblk(P, 256), 256, 0, s>>>(h->P, h->pnew, (const T*)h->pts_tmp, (T*)h->pts);
      e = cudaMemcpyAsync(h->pt_idx, ptx, O * 4, cudaMemcpyDeviceToDevice, s);
    }
    // internal orders: by point (new numbering), and by camera with the
    // points of each camera in increasing new index
    if (e == cudaSuccess) e = csr_build_async(h->pt_idx, h->O, h->P, h->perm_pt, h->rowptr_pt, scratch, derr, s);
    if (e == cudaSuccess) {
      k_gather_i32<<<nblk(O, 256), 256, 0, s>>>(h->O, h->perm_pt, h->cam_idx, key);
      e = csr_build_async(key, h->O, h->C, tmp, ptx, scratch, derr, s);
    }
    if (e == cudaSuccess) k_gather_i32<<<nblk(O, 256), 256, 0, s>>>(h->O, tmp, h->perm_pt, h->perm_cam);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    count_launch(5);
    cudaFree(scratch);
    cudaFree(key);
    cudaFree(tmp);
    cudaFree(ptx);
    CU(e);
  }

  // pieces: each camera's slots cut into runs of at most PIECE
  std::vector<int32_t> rp(C + 1);
  CU(cudaMemcpy(rp.data(), h->rowptr_cam, (C + 1) * 4, cudaMemcpyDeviceToHost));
  std::vector<int32_t> pc, pb, pe, cpp(C + 1);
  for (long long c = 0; c < C; ++c) {
    cpp[c] = (int32_t)pc.size();
    const int n = rp[c + 1] - rp[c];
    const int k = (n + PIECE - 1) / PIECE;
    for (int i = 0; i < k; ++i) {
      pc.push_back((int32_t)c);
      pb.push_back(rp[c] + (int)((long long)n * i / k));
      pe.push_back(rp[c] + (int)((long long)n * (i + 1) / k));
    }
  }
  cpp[C] = (int32_t)pc.size();
  h->npieces = (int)pc.size();
  CU(h->alloc(&h->piece_cam, pc.size() * 4));
  CU(h->alloc(&h->piece_beg, pc.size() * 4));
  CU(h->alloc(&h->piece_end, pc.size() * 4));
  CU(h->alloc(&h->cam_piece_ptr, (C + 1) * 4));
  CU(cudaMemcpy(h->piece_cam, pc.data(), pc.size() * 4, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(h->piece_beg, pb.data(), pb.size() * 4, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(h->piece_end, pe.data(), pe.size() * 4, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(h->cam_piece_ptr, cpp.data(), (C + 1) * 4, cudaMemcpyHostToDevice));

  // point chunks: runs of whole points with at most CHUNK_SLOTS observations
  // and CHUNK_PTS points (a point with more observations is a chunk alone)
  std::vector<int32_t> rq(P + 1), pch;
  {
    CU(cudaMemcpy(rq.data(), h->rowptr_pt, (P + 1) * 4, cudaMemcpyDeviceToHost));
    long long j = 0;
    while (j < P) {
      pch.push_back((int32_t)j);
      long long e = j + 1;
      while (e < P && e - j < CHUNK_PTS && rq[e + 1] - rq[j] <= CHUNK_SLOTS) ++e;
      j = e;
    }
    pch.push_back((int32_t)P);
    h->nchunks = (int)pch.size() - 1;
    CU(h->alloc(&h->pchunk, pch.size() * 4));
    CU(cudaMemcpy(h->pchunk, pch.data(), pch.size() * 4, cudaMemcpyHostToDevice));
  }
  if (lin_pt_smem<T>(true) > 48 * 1024)
    CU(cudaFuncSetAttribute(k_lin_pt<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lin_pt_smem<T>(true)));
  CU(cudaFuncSetAttribute(k_pass_fa<T, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fa_smem<T>(FA_CAMS)));
  CU(cudaFuncSetAttribute(k_pass_fa<T, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fa_smem<T>(FA_CAMS)));
  CU(cudaFuncSetAttribute(k_pass_fa<T, 0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, fa_smem<T>(FA_CAMS)));
  CU(cudaFuncSetAttribute(k_pass_fa<T, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, fa_smem<T>(FA_CAMS)));


  // observation data in both orders
  CU(h->alloc(&h->cm_pt, O * 4));
  CU(h->alloc(&h->pm_cam, O * 4));
  CU(h->alloc(&h->pm_pt, O * 4));
  CU(h->alloc(&h->cm_px, 2 * O * ts));
  CU(h->alloc(&h->pm_px, 2 * O * ts));
  k_gather_obs<T><<<nblk(O, 256), 256, 0, s>>>(h->O, h->perm_cam, h->perm_pt, h->cam_idx, h->pt_idx,
                                               (const T*)h->px_in, h->cm_pt, (T*)h->cm_px, h->pm_cam,
                                               h->pm_pt, (T*)h->pm_px);
  CU(h->alloc(&h->pm2cm, O * 4));
  {
    int32_t* inv = nullptr;
    CU(cudaMalloc(&inv, O * 4));
    k_invert_perm<<<nblk(O, 256), 256, 0, s>>>(h->O, h->perm_cam, inv);
    k_compose_perm<<<nblk(O, 256), 256, 0, s>>>(h->O, h->perm_pt, inv, h->pm2cm);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(inv);
    CU(e);
  }
  count_launch(3);

  // fused point-major pass A (both modes): every chunk's distinct cameras,
  // if no chunk has more than FA_CAMS of them
  {
    std::vector<int32_t> pmc(O), list, ptr(h->nchunks + 1), tmp;
    std::vector<int16_t> lc(O);
    CU(cudaMemcpy(pmc.data(), h->pm_cam, O * 4, cudaMemcpyDeviceToHost));
    bool ok = true;
    for (int k = 0; k < h->nchunks && ok; ++k) {
      const int s0 = rq[pch[k]], s1 = rq[pch[k + 1]];
      tmp.assign(pmc.begin() + s0, pmc.begin() + s1);
      std::sort(tmp.begin(), tmp.end());
      tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
      if ((int)tmp.size() > FA_CAMS) {
        ok = false;
        break;
      }
      ptr[k] = (int32_t)list.size();
      list.insert(list.end(), tmp.begin(), tmp.end());
      h->fa_nc = std::max(h->fa_nc, (int)tmp.size());
      for (int q = s0; q < s1; ++q)
        lc[q] = (int16_t)(std::lower_bound(tmp.begin(), tmp.end(), pmc[q]) - tmp.begin());
    }
    if (ok) {
      ptr[h->nchunks] = (int32_t)list.size();
      CU(h->alloc(&h->chunk_cams, std::max<size_t>(list.size(), 1) * 4));
      CU(h->alloc(&h->chunk_cam_ptr, ptr.size() * 4));
      CU(h->alloc(&h->pm_lc, O * 2));
      CU(cudaMemcpy(h->chunk_cams, list.data(), list.size() * 4, cudaMemcpyHostToDevice));
      CU(cudaMemcpy(h->chunk_cam_ptr, ptr.data(), ptr.size() * 4, cudaMemcpyHostToDevice));
      CU(cudaMemcpy(h->pm_lc, lc.data(), O * 2, cudaMemcpyHostToDevice));
      // per-chunk headers of the fused pass: j0, j1, s0, s1 | c0, nc, first
      // camera if the list is a contiguous range (else -1), 0
      std::vector<int4> hdr(2 * (size_t)h->nchunks);
      for (int k = 0; k < h->nchunks; ++k) {
        const int c0 = ptr[k], nc = ptr[k + 1] - ptr[k];
        const bool contiguous = nc > 0 && list[c0 + nc - 1] - list[c0] == nc - 1;
        hdr[2 * k] = make_int4(pch[k], pch[k + 1], rq[pch[k]], rq[pch[k + 1]]);
        hdr[2 * k + 1] = make_int4(c0, nc, contiguous ? list[c0] : -1, 0);
      }
      CU(h->alloc(&h->chunk_hdr, hdr.size() * sizeof(int4)));
      CU(cudaMemcpy(h->chunk_hdr, hdr.data(), hdr.size() * sizeof(int4), cudaMemcpyHostToDevice));
      h->fa = true;
    }
  }

  // linearisation and solver buffers
  CU(h->alloc(&h->camtab, CT * C * ts));
  CU(h->alloc(&h->ptab, 8 * P * ts));
  CU(h->alloc(&h->zbuf, 4 * O * ts));
  if (!h->mf) {
    CU(h->alloc(&h->Jcm, (size_t)NPLANE * O * ts));
    if (h->fa) {
      // the planes in point-major order for the fused stored pass A
      CU(h->alloc(&h->Jpm, (size_t)NPLANE * O * ts));
      if (fs_smem<T>(FA_CAMS) > 48 * 1024)
        CU(cudaFuncSetAttribute(k_pass_fs<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, fs_smem<T>(FA_CAMS)));
    }
  } else if (h->opt.huber_delta > 0) {
    CU(h->alloc(&h->cm_sw, O * ts));
    CU(h->alloc(&h->pm_sw, O * ts));
  }
  CU(h->alloc(&h->U, 45 * C * 8));
  CU(h->alloc(&h->gc, 9 * C * 8));
  CU(h->alloc(&h->V, 6 * P * 8));
  CU(h->alloc(&h->gp, 3 * P * 8));
  CU(h->alloc(&h->Vinv, 6 * P * ts));
  CU(h->alloc(&h->y0, 3 * P * ts));
  CU(h->alloc(&h->Minv, 45 * C * 8));
  CU(h->alloc(&h->x, 9 * C * 8));
  CU(h->alloc(&h->r, 9 * C * 8));
  CU(h->alloc(&h->z, 9 * C * 8));
  CU(h->alloc(&h->p, 9 * C * 8));
  CU(h->alloc(&h->q, 9 * C * 8));
  CU(h->alloc(&h->pT, PV * C * ts));
  CU(h->alloc(&h->xT, PV * C * ts));
  CU(cudaMemsetAsync(h->ptab, 0, 8 * P * ts, s));
  CU(h->alloc(&h->dp, 3 * P * ts));
  CU(h->alloc(&h->part, (size_t)PART * std::max(h->npieces, 1) * 8));
  h->ncb = (int)nblk(C, CAM_THREADS);
  if (h->opt.solver == BA_SOLVER_CHOLESKY) {
    // the direct solve: W of every observation; partial copies of S, one
    // CTA per camera and copy building them (as many copies as keep every
    // CTA resident and fit in 96 MB, so in L2; at most 8, at least 1); the
    // band tiles of the whole lower triangle; the factorisation's task list
    // (ba_band_sched.h) for one block per SM
    const size_t n = 9 * (size_t)C;
    int dev = 0, nsm = 1, occ = 1;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_schur_dense<double>, DENSE_THREADS, 0));
    const size_t by_slots = (size_t)std::max(1, occ) * (size_t)nsm / (size_t)std::max<long long>(1, C);
    const size_t by_bytes = (96ull << 20) / (n * n * 8);
    h->nseg = (int)std::max<size_t>(1, std::min<size_t>(8, std::min(by_slots, by_bytes)));
    CU(h->alloc(&h->Wd, 27ull * 8 * (size_t)std::max<long long>(O, 1)));
    CU(h->alloc(&h->Spart, (size_t)h->nseg * n * n * 8));
    h->bnb = (int)((n + BAND_TB - 1) / BAND_TB);
    h->bwt = h->bnb - 1;
    const long long nupd = (long long)h->bnb * h->bwt * (h->bwt + 1) / 2;
    const int s_upd = (int)std::max(1LL, (nupd + (4LL << 20) - 1) / (4LL << 20));
    h->band_grid = std::max(1, nsm);
    h->band_crit = h->band_grid >= 2 ? std::min(BAND_CRIT_BLOCKS, std::max(1, h->band_grid / 8)) : 0;
    const std::vector<BandTask> tasks = band_tasks(h->bnb, h->bwt, s_upd, h->band_grid, h->band_crit, &h->bncrit);
    static_assert(sizeof(BandTask) == sizeof(int4), "a task is read as an int4");
    if (h->bncrit == 0) h->band_crit = 0;
    h->bntask = (int)tasks.size();
    h->bT_bytes = (size_t)h->bnb * (h->bwt + 1) * (BAND_TB * BAND_TB) * sizeof(double);
    h->bflag_count = 2 * (size_t)h->bnb * (h->bwt + 1) + 6 + h->bnb;
    CU(h->alloc(&h->bT, h->bT_bytes));
    CU(h->alloc(&h->brs, 8ull * h->bnb * BAND_TB));
    CU(h->alloc(&h->bUi, 8ull * h->bnb * BAND_TB * BAND_TB));
    CU(h->alloc(&h->dy, 8ull * h->bnb * BAND_TB));
    CU(h->alloc(&h->bflag, sizeof(int) * h->bflag_count));
    CU(h->alloc(&h->btask, sizeof(int4) * tasks.size()));
    CU(cudaMemcpy(h->btask, tasks.data(), sizeof(int4) * tasks.size(), cudaMemcpyHostToDevice));
  }
  h->npb = (int)nblk(P, PT_THREADS);
  CU(h->alloc(&h->dot_pq, h->ncb * 8));
  CU(h->alloc(&h->dot_rz, 2 * h->ncb * 8));
  CU(h->alloc(&h->dot_rr, h->ncb * 8));
  CU(h->alloc(&h->dot_bb, h->ncb * 8));
  CU(h->alloc(&h->dot_gc, h->ncb * 8));
  CU(h->alloc(&h->dot_gp, std::max(h->nchunks, 1) * 8));
  h->cap = h->opt.max_stats;
  CU(h->alloc(&h->stats, (size_t)h->cap * sizeof(ba_iter_stats)));
  CU(cudaMemsetAsync(h->stats, 0, (size_t)h->cap * sizeof(ba_iter_stats), s));
  CU(cudaMemsetAsync(h->x, 0, 9 * C * 8, s));
  CU(cudaMemsetAsync(h->dp, 0, 3 * P * ts, s));
  CU(cudaMemsetAsync(h->xT, 0, PV * C * ts, s));

  if (h->mf) enqueue_cost<T, true>(h);
  else enqueue_cost<T, false>(h);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(&err, &h->st->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (err & 2) return fail(BA_ERR_NONFINITE, "non-finite initial cost");
  return BA_OK;
}

// The stale cost, before a call reads F on the host.
ba_status settle_cost(ba_problem* h) {
  if (!h->cost_pending) return BA_OK;
  BA_DISPATCH(h, enqueue_cost, true);
  CU(cudaGetLastError());
  h->cost_pending = false;
  return BA_OK;
}

ba_status set_flag(ba_problem* h, size_t offset, int value) {
  // write one int of DevState, stream-ordered
  k_set_int<<<1, 32, 0, h->s>>>(reinterpret_cast<int*>(reinterpret_cast<char*>(h->st) + offset), value);
  count_launch();
  CU(cudaGetLastError());
  return BA_OK;
}

// Copy caller-ordered points (any memory) into parameter buffer `buf`.
// Cameras (cams_tmp) or points (pts_tmp, caller's order) into (store) or out
// of the current parameter buffer.
void params_cur(ba_problem* h, bool cams, bool points, bool store = true) {
  if (cams) {
    const long long n = 9LL * h->C;
    if (h->prec == BA_PREC_F32)
      k_cams_cur<float><<<nblk(n, 256), 256, 0, h->s>>>(n, h->st, (const float*)h->cams_tmp, (float*)h->cams,
                                                         store ? 1 : 0);
    else
      k_cams_cur<double><<<nblk(n, 256), 256, 0, h->s>>>(n, h->st, (const double*)h->cams_tmp, (double*)h->cams,
                                                          store ? 1 : 0);
    count_launch();
  }
  if (points) {
    const int32_t* idx = store ? h->pnew : h->pnewpos;
    if (h->prec == BA_PREC_F32)
      k_points_cur<float><<<nblk(h->P, 256), 256, 0, h->s>>>(h->P, idx, h->st, (float*)h->pts_tmp, (float*)h->pts,
                                                             store ? 1 : 0);
    else
      k_points_cur<double><<<nblk(h->P, 256), 256, 0, h->s>>>(h->P, idx, h->st, (double*)h->pts_tmp,
                                                              (double*)h->pts, store ? 1 : 0);
    count_launch();
  }
}

ba_status load_points(ba_problem* h, const void* points, int buf) {
  const size_t pb = 3ull * h->P * h->tsize;
  CU(cudaMemcpyAsync(h->pts_tmp, points, pb, cudaMemcpyDefault, h->s));
  void* dst = (char*)h->pts + buf * pb;
  if (h->prec == BA_PREC_F32)
    k_gather_rows<float, 3><<<nblk(h->P, 256), 256, 0, h->s>>>(h->P, h->pnew, (const float*)h->pts_tmp,
                                                               (float*)dst);
  else
    k_gather_rows<double, 3><<<nblk(h->P, 256), 256, 0, h->s>>>(h->P, h->pnew, (const double*)h->pts_tmp,
                                                                (double*)dst);
  count_launch();
  CU(cudaGetLastError());
  return BA_OK;
}

ba_status set_probe_lambda(ba_problem* h, double lam) {
  CU(cudaMemcpyAsync(&h->st->lam_probe, &lam, sizeof(double), cudaMemcpyHostToDevice, h->s));
  CU(cudaStreamSynchronize(h->s));
  return BA_OK;
}

// Features, scaled inverse factors and probe products S^ z^ at the current
// parameters and damping *lam_ptr (ba_learn_collect).
template <typename T, bool MF>
void enqueue_collect(ba_problem* h, const double* lam_ptr, int K, const float* zhat, float* X, float* Ahat,
                     float* Yhat) {
  cudaStream_t s = h->s;
  const double dmin = h->opt.diag_min, dmax = h->opt.diag_max;
  enqueue_lin<T, MF>(h, 1);
  k_pt_damp<T><<<nblk(h->P, PT_THREADS), PT_THREADS, 0, s>>>(h->P, h->V, h->gp, lam_ptr, dmin, dmax, (T*)h->Vinv,
                                                            (T*)h->y0);
  k_schur_cam<T, MF><<<h->npieces, LIN_THREADS, 0, s>>>(
      h->piece_cam, h->piece_beg, h->piece_end, h->cm_pt, (const T*)h->Jcm, (const T*)h->camtab, (const T*)h->pts,
      (const T*)h->cm_sw, h->st, h->P, (const T*)h->Vinv, (const T*)h->y0, h->O, h->part);
  k_cam_combine_schur<T, MF><<<h->ncb, CAM_THREADS, 0, s>>>(
      h->C, h->cam_piece_ptr, h->part, h->U, h->gc, (const T*)h->camtab, lam_ptr, dmin, dmax, h->Minv, h->x, h->r,
      h->z, h->p, (T*)h->pT, h->dot_rz + h->ncb, h->dot_bb, h->fixed, h->st, h->Sii);
  enqueue_coupling<T, MF>(h, lam_ptr);
  k_learn_features<<<h->ncb, CAM_THREADS, 0, s>>>(h->C, h->Sii, h->U, lam_ptr, dmin, dmax, h->rowptr_cam, X, Ahat,
                                                  h->Dsc, h->kap);
  count_launch(4);
  for (int k = 0; k < K; ++k) {
    k_probe_in<T, MF><<<nblk(h->C, 128), 128, 0, s>>>(h->C, K, k, zhat, h->Dsc, (const T*)h->camtab, h->p,
                                                      (T*)h->pT);
    enqueue_schur_product<T, MF>(h, (const T*)h->pT, -1, 0);
    k_pcg_q<T, MF><<<h->ncb, VT, 0, s>>>(h->C, h->cam_piece_ptr, h->part, h->U, (const T*)h->camtab, lam_ptr, dmin,
                                        dmax, h->p, h->q, nullptr, h->fixed, h->st, 0);
    k_probe_out<<<nblk(h->C, 128), 128, 0, s>>>(h->C, K, k, h->q, h->Dsc, Yhat);
    count_launch(3);
  }
}

// Slow-mode probes: z^_j = D^{1/2} (x_ref - x_its[j]) / rms, x_ref from a
// PCG run of maxiter_ref iterations / tol_ref, x_k after k iterations.
template <typename T, bool MF>
void enqueue_slow_probes(ba_problem* h, const double* lam_ptr, int n, const int* its, int maxiter_ref, double tol_ref,
                         float* zhat, double* xref) {
  cudaStream_t s = h->s;
  enqueue_collect<T, MF>(h, lam_ptr, 0, nullptr, h->Xf, nullptr, nullptr);  // scales D
  enqueue_solve<T, MF>(h, lam_ptr, maxiter_ref, tol_ref, false, 16);
  cudaMemcpyAsync(xref, h->x, 72ull * h->C, cudaMemcpyDeviceToDevice, s);
  for (int j = 0; j < n; ++j) {
    enqueue_solve<T, MF>(h, lam_ptr, its[j], 0.0, false);
    k_slow_diff<<<nblk(9LL * h->C, 256), 256, 0, s>>>(h->C, n, j, xref, h->x, h->Dsc, zhat);
    count_launch();
  }
  k_slow_normalize<<<1, 256, 0, s>>>(h->C, n, zhat);
  count_launch();
}

ba_status ensure_learn_buffers(ba_problem* h) {
  if (h->Sii) return BA_OK;
  CU(h->alloc(&h->mlp, (size_t)MLP_NPARAM * 4));
  CU(h->alloc(&h->Sii, 45ull * h->C * 8));
  CU(h->alloc(&h->Xf, (size_t)MLP_FIN * h->C * 4));
  CU(h->alloc(&h->Ef, (size_t)MLP_FOUT * h->C * 4));
  CU(h->alloc(&h->Dsc, 9ull * h->C * 8));
  CU(h->alloc(&h->kap, (size_t)h->C * 8));
  CU(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_SMEM_FWD));
  return BA_OK;
}

}  // namespace

static __global__ void k_f2d(long long n, const float* __restrict__ a, double* __restrict__ b) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}
static __global__ void k_d2f(long long n, const double* __restrict__ a, float* __restrict__ b) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

extern "C" ba_status ba_backward(ba_problem* h, double lambda, int maxiter, double tol, const void* dL_dcams,
                                 const void* dL_dpoints, void* dL_dpixels_out, void* dL_dcams0_out,
                                 void* dL_dpoints0_out, int* iters, double* rel_res, void* stream);

// The adjoint of an FP32 problem, solved in FP64.  Its system H v = dL/dtheta
// is ill-conditioned and its implicit Schur product cancels (measured on the
// 64-camera workload: condition ~5.5e3 after block-Jacobi scaling, |U* v| /
// |S v| ~ 190), which would turn FP32 rounding of the Jacobian into ~1e-2
// relative gradient errors.  So the first call builds an FP64 twin of the
// problem (the same observations; the FP32 parameters and pixels promoted,
// exactly), later calls refresh its parameters, pixels and frozen mask, and
// the twin's FP64 adjoint is returned in FP32.  Scratch is allocated per call.
ba_status backward_via_f64(ba_problem* h, double lambda, int maxiter, double tol, const float* dLc,
                           const float* dLp, float* dpix_out, float* dc0_out, float* dp0_out, int* iters,
                           double* rel_res, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const long long C = h->C, P = h->P, O = h->O;
  std::vector<void*> tmp;
  auto grab = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    tmp.push_back(p);
    return p;
  };
  auto release = [&]() {
    cudaStreamSynchronize(s);
    for (void* p : tmp) cudaFree(p);
  };
  float* c32 = (float*)grab(9 * C * 4);
  float* p32 = (float*)grab(3 * P * 4);
  double* c64 = (double*)grab(9 * C * 8);
  double* p64 = (double*)grab(3 * P * 8);
  double* x64 = (double*)grab(2 * O * 8);
  double* gc64 = dLc ? (double*)grab(9 * C * 8) : nullptr;
  double* gp64 = dLp ? (double*)grab(3 * P * 8) : nullptr;
  double* px64 = (double*)grab(2 * O * 8);
  double* dc64 = dc0_out ? (double*)grab(9 * C * 8) : nullptr;
  double* dp64 = dp0_out ? (double*)grab(3 * P * 8) : nullptr;
  int32_t* ptc = (int32_t*)grab(O * 4);
  if (!c32 || !p32 || !c64 || !p64 || !x64 || (dLc && !gc64) || (dLp && !gp64) || !px64 || (dc0_out && !dc64) ||
      (dp0_out && !dp64) || !ptc) {
    release();
    return fail(BA_ERR_OOM, "scratch of the FP64 adjoint");
  }
  ba_status st = ba_get_params(h, c32, p32, stream);
  if (st == BA_OK) {
    // (ordered after the problem's stream by ba_get_params)
    k_f2d<<<nblk(9 * C, 256), 256, 0, s>>>(9 * C, c32, c64);
    k_f2d<<<nblk(3 * P, 256), 256, 0, s>>>(3 * P, p32, p64);
    k_f2d<<<nblk(2 * O, 256), 256, 0, s>>>(2 * O, (const float*)h->px_in, x64);
    k_gather_i32<<<nblk(O, 256), 256, 0, s>>>((int)O, h->pt_idx, h->pnew, ptc);  // the caller's point numbering
    if (dLc) k_f2d<<<nblk(9 * C, 256), 256, 0, s>>>(9 * C, dLc, gc64);
    if (dLp) k_f2d<<<nblk(3 * P, 256), 256, 0, s>>>(3 * P, dLp, gp64);
    count_launch(4 + (dLc ? 1 : 0) + (dLp ? 1 : 0));
    if (cudaGetLastError() != cudaSuccess) st = fail(BA_ERR_CUDA, "promotion kernels failed");
  }
  if (st == BA_OK && !h->twin) {
    ba_options o = h->opt;
    o.precision = BA_PREC_F64;
    o.jacobian_mode = BA_JAC_AUTO;
    o.solver = BA_SOLVER_PCG;
    st = ba_problem_create(&h->twin, (int)C, (int)P, (int)O, c64, p64, h->cam_idx, ptc, x64, &o, stream);
  } else if (st == BA_OK) {
    st = ba_set_params(h->twin, c64, p64, stream);
    if (st == BA_OK) st = ba_set_pixels(h->twin, x64, stream);
  }
  if (st == BA_OK) st = ba_set_fixed(h->twin, h->fixed, stream);
  if (st == BA_OK)
    st = ba_backward(h->twin, lambda, maxiter, tol, gc64, gp64, px64, dc64, dp64, iters, rel_res, stream);
  if (st == BA_OK) {
    k_d2f<<<nblk(2 * O, 256), 256, 0, s>>>(2 * O, px64, dpix_out);
    if (dc0_out) k_d2f<<<nblk(9 * C, 256), 256, 0, s>>>(9 * C, dc64, dc0_out);
    if (dp0_out) k_d2f<<<nblk(3 * P, 256), 256, 0, s>>>(3 * P, dp64, dp0_out);
    count_launch(1 + (dc0_out ? 1 : 0) + (dp0_out ? 1 : 0));
    if (cudaGetLastError() != cudaSuccess) st = fail(BA_ERR_CUDA, "conversion kernels failed");
  }
  release();
  return st;
}

extern "C" {

ba_status ba_options_default(ba_options* o) {
  if (!o) return fail(BA_ERR_INVALID_ARG, "NULL options");
  o->precision = BA_PREC_F64;
  o->huber_delta = 0.0;
  o->lambda0 = 1e-4;
  o->up = 2.0;
  o->down = 0.0625;
  o->rho_good = 0.75;
  o->rho_bad = 0.25;
  o->lambda_min = 1e-16;
  o->lambda_max = 1e32;
  o->diag_min = 1e-6;
  o->diag_max = 1e32;
  o->pcg_maxiter = 250;
  o->pcg_tol = 1e-4;
  o->use_graph = 1;
  o->max_stats = 4096;
  o->jacobian_mode = BA_JAC_AUTO;
  o->solver = BA_SOLVER_PCG;
  return BA_OK;
}

ba_status ba_problem_create(ba_problem** out, int C, int P, int O, const void* cams, const void* points,
                            const int32_t* cam_idx, const int32_t* pt_idx, const void* pixels,
                            const ba_options* opt, void* stream) {
  if (!out) return fail(BA_ERR_INVALID_ARG, "NULL output handle");
  *out = nullptr;
  if (C < 1 || P < 1 || O < 1) return fail(BA_ERR_INVALID_ARG, "C, P and O must be >= 1 (got %d, %d, %d)", C, P, O);
  if (!cams || !points || !cam_idx || !pt_idx || !pixels) return fail(BA_ERR_INVALID_ARG, "NULL input array");
  ba_options o;
  if (opt) o = *opt;
  else ba_options_default(&o);
  ba_status st = check_options(&o);
  if (st != BA_OK) return st;
  if (o.solver == BA_SOLVER_CHOLESKY && 9LL * C > BA_DENSE_MAX_DIM)
    return fail(BA_ERR_INVALID_ARG, "BA_SOLVER_CHOLESKY needs 9C <= %d (C = %d)", BA_DENSE_MAX_DIM, C);
  ba_problem* h = new (std::nothrow) ba_problem();
  if (!h) return fail(BA_ERR_OOM, "host allocation failed");
  h->C = C;
  h->P = P;
  h->O = O;
  h->prec = o.precision;
  h->mf = o.jacobian_mode == BA_JAC_RECOMPUTE || (o.jacobian_mode == BA_JAC_AUTO && o.precision == BA_PREC_F32);
  h->tsize = o.precision == BA_PREC_F32 ? 4 : 8;
  h->opt = o;
  cudaError_t e = cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    delete h;
    return fail(BA_ERR_CUDA, "stream/event creation failed: %s", cudaGetErrorString(e));
  }
  st = enter(h, stream);
  if (st == BA_OK) {
    st = h->prec == BA_PREC_F32 ? create_impl<float>(h, cams, points, cam_idx, pt_idx, pixels)
                                : create_impl<double>(h, cams, points, cam_idx, pt_idx, pixels);
  }
  if (st != BA_OK) {
    std::string msg = g_err;
    cudaStreamSynchronize(h->s);
    delete h;
    g_err = msg;
    return st;
  }
  *out = h;
  return BA_OK;
}

ba_status ba_problem_destroy(ba_problem* h) {
  if (!h) return BA_OK;
  cudaStreamSynchronize(h->s);
  delete h;
  return BA_OK;
}

ba_status ba_lm_step(ba_problem* h, void* stream) {
  // one trial: a replay of the captured trial graph (as ba_solve(1))
  return ba_solve(h, 1, stream);
}

ba_status ba_solve(ba_problem* h, int iters, void* stream) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "NULL problem");
  if (iters < 0) return fail(BA_ERR_INVALID_ARG, "iters < 0");
  ba_status st = enter(h, stream);
  if (st != BA_OK) return st;
  if (iters > 0) h->cost_pending = false;  // every trial starts with the stale cost
  if (h->xch) {
    // a part of a point-partitioned problem: direct launches, the caller's
    // all-reduce at each exchange
    h->xerr = 0;
    for (int i = 0; i < iters && !h->xerr; ++i) enqueue_trial_any(h);
    CU(cudaGetLastError());
    if (h->xerr)
      return fail(BA_ERR_CUDA, h->xerr == 2 ? "the exchange callback failed" : "exchange buffer too small or copy failed");
    return leave(h, stream);
  }
  // the direct solver's factorisation is a cooperative launch: its trials
  // run as direct launches
  if (!h->opt.use_graph || h->opt.solver == BA_SOLVER_CHOLESKY) {
    for (int i = 0; i < iters; ++i) enqueue_trial_any(h);
    CU(cudaGetLastError());
    return leave(h, stream);
  }
  if (!h->gexec && iters > 0) {
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
    ba::g_capturing = true;
    enqueue_trial_any(h);
    ba::g_capturing = false;
    cudaError_t e = cudaStreamEndCapture(h->s, &g);
    if (e != cudaSuccess) return fail(BA_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    size_t n = 0;
    cudaGraphGetNodes(g, nullptr, &n);
    h->gnodes = n;
    e = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      h->gexec = nullptr;
      return fail(BA_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
  }
  for (int i = 0; i < iters; ++i) {
    CU(cudaGraphLaunch(h->gexec, h->s));
    count_launch(h->gnodes);
  }
  return leave(h, stream);
}

ba_status ba_get_params(ba_problem* h, void* cams_out, void* points_out, void* stream) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "NULL problem");
  ba_status st = enter(h, stream);
  if (st != BA_OK) return st;
  // from the current buffer (its index read on the device), points back to
  // the caller's order
  const size_t cb = 9ull * h->C * h->tsize, pb = 3ull * h->P * h->tsize;
  if (cams_out) {
    params_cur(h, true, false, false);
    CU(cudaMemcpyAsync(cams_out, h->cams_tmp, cb, cudaMemcpyDefault, h->s));
  }
  if (points_out) {
    params_cur(h, false, true, false);
    CU(cudaMemcpyAsync(points_out, h->pts_tmp, pb, cudaMemcpyDefault, h->s));
  }
  return leave(h, stream);
}

ba_status ba_set_params(ba_problem* h, const void* cams, const void* points, void* stream) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "NULL problem");
  ba_status st = enter(h, stream);
  if (st != BA_OK) return st;
  // into the current buffer, its index read on the device (no host round trip)
  const size_t cb = 9ull * h->C * h->tsize, pb = 3ull * h->P * h->tsize;
  if (cams) {
    CU(cudaMemcpyAsync(h->cams_tmp, cams, cb, cudaMemcpyDefault, h->s));
    params_cur(h, true, false);
  }
  if (points) {
    CU(cudaMemcpyAsync(h->pts_tmp, points, pb, cudaMemcpyDefault, h->s));
    params_cur(h, false, true);
  }
  st = set_flag(h, offsetof(DevState, need_lin), 1);
  if (st != BA_OK) return st;
  // F is evaluated lazily: by the next trial, or by a call that reads it
  st = set_flag(h, offsetof(DevState, need_cost), 1);
  if (st != BA_OK) return st;
  h->cost_pending = true;
  return leave(h, stream);
}

ba_status ba_set_pixels(ba_problem* h, const void* pixels, void* stream) {
  if (!h || !pixels) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  ba_status st = enter(h, stream);
  if (st != BA_OK) return st;
  CU(cudaMemcpyAsync(h->px_in, pixels, 2ull * h->O * h->tsize, cudaMemcpyDefault, h->s));
  if (h->prec == BA_PREC_F32)
    k_gather_obs<float><<<nblk(h->O, 256), 256, 0, h->s>>>(h->O, h->perm_cam, h->perm_pt, h->cam_idx, h->pt_idx,
                                                           (const float*)h->px_in, h->cm_pt, (float*)h->cm_px,
                                                           h->pm_cam, h->pm_pt, (float*)h->pm_px);
  else
    k_gather_obs<double><<<nblk(h->O, 256), 256, 0, h->s>>>(h->O, h->perm_cam, h->perm_pt, h->cam_idx,
                                                            h->pt_idx, (const double*)h->px_in, h->cm_pt,
                                                            (double*)h->cm_px, h->pm_cam, h->pm_pt,
                                                            (double*)h->pm_px);
  count_launch();
  st = set_flag(h, offsetof(DevState, need_lin), 1);
  if (st != BA_OK) return st;
  // F is evaluated lazily: by the next trial, or by a call that reads it
  st = set_flag(h, offsetof(DevState, need_cost), 1);
  if (st != BA_OK) return st;
  h->cost_pending = true;
  return leave(h, stream);
}

ba_status ba_get_stats(ba_problem* h, ba_iter_stats* host_out, int cap, int* n_out) {
  if (!h || (cap > 0 && !host_out)) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  DevState ds;
  CU(cudaMemcpyAsync(&ds, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->s));
  CU(cudaStreamSynchronize(h->s));
  const long long avail = std::min<long long>(ds.trials, h->cap);
  const long long n = std::min<long long>(avail, cap > 0 ? cap : 0);
  for (long long i = 0; i < n; ++i) {
    const long long t = ds.trials - n + i;
    CU(cudaMemcpy(host_out + i, h->stats + (t % h->cap), sizeof(ba_iter_stats), cudaMemcpyDeviceToHost));
  }
  if (n_out) *n_out = (int)n;
  if (ds.nonfinite > 0) {
    ba_status st = set_flag(h, offsetof(DevState, nonfinite), 0);
    if (st != BA_OK) return st;
    return fail(BA_ERR_NONFINITE, "%d trial(s) produced a non-finite cost and were rejected", ds.nonfinite);
  }
  return BA_OK;
}

ba_status ba_get_scalars(ba_problem* h, double* cost, double* lambda) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "NULL problem");
  ba_status st0 = settle_cost(h);
  if (st0 != BA_OK) return st0;
  DevState ds;
  CU(cudaMemcpyAsync(&ds, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->s));
  CU(cudaStreamSynchronize(h->s));
  if (cost) *cost = ds.F;
  if (lambda) *lambda = ds.lam;
  return BA_OK;
}

ba_status ba_set_lambda(ba_problem* h, double lambda) {
  if (!h || !(lambda > 0)) return fail(BA_ERR_INVALID_ARG, "lambda must be > 0");
  CU(cudaMemcpyAsync(&h->st->lam, &lambda, sizeof(double), cudaMemcpyHostToDevice, h->s));
  CU(cudaStreamSynchronize(h->s));
  return BA_OK;
}

size_t ba_state_size(const ba_problem* h) { return h ? 9ull * h->C + 3ull * h->P + 4 : 0; }

ba_status ba_get_state(ba_problem* h, double* out) {
  if (!h || !out) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  ba_status st0 = settle_cost(h);
  if (st0 != BA_OK) return st0;
  DevState ds;
  CU(cudaMemcpyAsync(&ds, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->s));
  CU(cudaStreamSynchronize(h->s));
  const size_t nc = 9ull * h->C, np = 3ull * h->P;
  std::vector<char> buf((nc + np) * h->tsize);
  ba_status st = ba_get_params(h, buf.data(), buf.data() + nc * h->tsize, h->s);
  if (st != BA_OK) return st;
  CU(cudaStreamSynchronize(h->s));
  for (size_t i = 0; i < nc + np; ++i)
    out[i] = h->prec == BA_PREC_F32 ? (double)((float*)buf.data())[i] : ((double*)buf.data())[i];
  out[nc + np] = ds.F;
  out[nc + np + 1] = ds.lam;
  out[nc + np + 2] = (double)ds.trials;
  out[nc + np + 3] = (double)ds.need_lin;
  return BA_OK;
}

ba_status ba_set_state(ba_problem* h, const double* in) {
  if (!h || !in) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  const size_t nc = 9ull * h->C, np = 3ull * h->P;
  std::vector<char> buf((nc + np) * h->tsize);
  for (size_t i = 0; i < nc + np; ++i) {
    if (h->prec == BA_PREC_F32) ((float*)buf.data())[i] = (float)in[i];
    else ((double*)buf.data())[i] = in[i];
  }
  DevState ds;
  CU(cudaMemcpyAsync(&ds, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->s));
  CU(cudaStreamSynchronize(h->s));
  CU(cudaMemcpy((char*)h->cams + ds.cur * nc * h->tsize, buf.data(), nc * h->tsize, cudaMemcpyHostToDevice));
  ba_status st = load_points(h, buf.data() + nc * h->tsize, ds.cur);
  if (st != BA_OK) return st;
  CU(cudaStreamSynchronize(h->s));
  ds.F = in[nc + np];
  ds.lam = in[nc + np + 1];
  ds.trials = (long long)in[nc + np + 2];
  ds.need_lin = 1;
  ds.nonfinite = 0;
  CU(cudaMemcpy(h->st, &ds, sizeof(DevState), cudaMemcpyHostToDevice));
  return BA_OK;
}

const char* ba_last_error(void) { return g_err.c_str(); }

ba_status ba_get_csr(ba_problem* h, int32_t* perm_cam, int32_t* rowptr_cam, int32_t* perm_pt, int32_t* rowptr_pt,
                     void* stream) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "NULL problem");
  ba_status st = enter(h, stream);
  if (st != BA_OK) return st;
  if (perm_cam) CU(cudaMemcpyAsync(perm_cam, h->xperm_cam, 4ull * h->O, cudaMemcpyDeviceToDevice, h->s));
  if (rowptr_cam) CU(cudaMemcpyAsync(rowptr_cam, h->rowptr_cam, 4ull * (h->C + 1), cudaMemcpyDeviceToDevice, h->s));
  if (perm_pt) CU(cudaMemcpyAsync(perm_pt, h->xperm_pt, 4ull * h->O, cudaMemcpyDeviceToDevice, h->s));
  if (rowptr_pt) CU(cudaMemcpyAsync(rowptr_pt, h->xrowptr_pt, 4ull * (h->P + 1), cudaMemcpyDeviceToDevice, h->s));
  return leave(h, stream);
}

ba_status ba_linearize(ba_problem* h, double* U, double* V, double* gc, double* gp, void* Jc, void* Jp, void* w,
                       void* stream) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "NULL problem");
  ba_status st = enter(h, stream);
  if (st != BA_OK) return st;
  st = set_flag(h, offsetof(DevState, need_lin), 1);
  if (st != BA_OK) return st;
  BA_DISPATCH(h, enqueue_lin, 1);
  if (Jc || Jp || w) BA_DISPATCH(h, launch_export, Jc, Jp, w);
  if (U) k_unpack_sym<<<nblk(81ll * h->C, 256), 256, 0, h->s>>>(h->C, 9, h->U, nullptr, U);
  if (V) k_unpack_sym<<<nblk(9ll * h->P, 256), 256, 0, h->s>>>(h->P, 3, h->V, h->pnewpos, V);
  if (gc) CU(cudaMemcpyAsync(gc, h->gc, 72ull * h->C, cudaMemcpyDeviceToDevice, h->s));
  if (gp) k_gather_rows<double, 3><<<nblk(h->P, 256), 256, 0, h->s>>>(h->P, h->pnewpos, h->gp, gp);
  count_launch(3);
  CU(cudaGetLastError());
  return leave(h, stream);
}

ba_status ba_schur_matvec(ba_problem* h, double lambda, const double* x, double* y, void* stream) {
  if (!h || !x || !y) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  ba_status st = enter(h, stream);
  if (st != BA_OK) return st;
  st = set_probe_lambda(h, lambda);
  if (st != BA_OK) return st;
  const double* lp = &h->st->lam_probe;
  CU(cudaMemcpyAsync(h->p, x, 72ull * h->C, cudaMemcpyDeviceToDevice, h->s));
  BA_DISPATCH(h, enqueue_lin, 1);
  BA_DISPATCH(h, enqueue_matvec, lp);
  CU(cudaMemcpyAsync(y, h->q, 72ull * h->C, cudaMemcpyDeviceToDevice, h->s));
  CU(cudaGetLastError());
  return leave(h, stream);
}

ba_status ba_damped_solve(ba_problem* h, double lambda, int maxiter, double tol, double* dc, void* dp, int* iters,
                          double* rel_res, void* stream) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "NULL problem");
  if (maxiter < 0 || maxiter > 100000 || !(tol >= 0)) return fail(BA_ERR_INVALID_ARG, "bad maxiter/tol");
  ba_status st = enter(h, stream);
  if (st != BA_OK) return st;
  st = set_probe_lambda(h, lambda);
  if (st != BA_OK) return st;
  const double* lp = &h->st->lam_probe;
  BA_DISPATCH(h, enqueue_lin, 1);
  BA_DISPATCH(h, enqueue_solve, lp, maxiter, tol, h->learned, 16);
  CU(cudaGetLastError());
  if (dc) CU(cudaMemcpyAsync(dc, h->x, 72ull * h->C, cudaMemcpyDeviceToDevice, h->s));
  if (dp) {
    if (h->prec == BA_PREC_F32)
      k_gather_rows<float, 3><<<nblk(h->P, 256), 256, 0, h->s>>>(h->P, h->pnewpos, (const float*)h->dp, (float*)dp);
    else
      k_gather_rows<double, 3><<<nblk(h->P, 256), 256, 0, h->s>>>(h->P, h->pnewpos, (const double*)h->dp,
                                                                  (double*)dp);
  }
  DevState ds;
  CU(cudaMemcpyAsync(&ds, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->s));
  CU(cudaStreamSynchronize(h->s));
  if (iters) *iters = ds.pcg_iters;
  if (rel_res) *rel_res = ds.pcg_rel;
  return leave(h, stream);
}

ba_status ba_project(int precision, int C, int P, int O, const void* cams, const void* points,
                     const int32_t* cam_idx, const int32_t* pt_idx, void* out, void* stream) {
  if (C < 1 || P < 1 || O < 0) return fail(BA_ERR_INVALID_ARG, "bad sizes");
  if (O == 0) return BA_OK;
  if (!cams || !points || !cam_idx || !pt_idx || !out) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == BA_PREC_F32)
    k_project<float><<<nblk(O, 256), 256, 0, s>>>(O, (const float*)cams, (const float*)points, cam_idx, pt_idx,
                                                  (float*)out);
  else if (precision == BA_PREC_F64)
    k_project<double><<<nblk(O, 256), 256, 0, s>>>(O, (const double*)cams, (const double*)points, cam_idx, pt_idx,
                                                   (double*)out);
  else
    return fail(BA_ERR_INVALID_ARG, "bad precision");
  count_launch();
  CU(cudaGetLastError());
  return BA_OK;
}

ba_status ba_csr_build(const int32_t* keys, int n, int n_keys, int32_t* perm_out, int32_t* rowptr_out,
                       void* stream) {
  if (n < 0 || n_keys < 1) return fail(BA_ERR_INVALID_ARG, "n must be >= 0 and n_keys >= 1");
  if ((n > 0 && (!keys || !perm_out)) || !rowptr_out) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  void* scratch = nullptr;
  CU(cudaMalloc(&scratch, ba::csr_scratch_bytes(n)));
  int* d_err = reinterpret_cast<int*>(static_cast<char*>(scratch) + ba::csr_scratch_bytes(n) - 256);
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = ba::csr_build_async(keys, n, n_keys, perm_out, rowptr_out, scratch, d_err, s);
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(scratch);
  if (e != cudaSuccess) return fail(BA_ERR_CUDA, "csr build failed: %s", cudaGetErrorString(e));
  if (err) return fail(BA_ERR_INVALID_ARG, "key out of range [0, %d)", n_keys);
  return BA_OK;
}

ba_status ba_set_fixed(ba_problem* h, const uint8_t* mask, void* stream) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "NULL problem");
  ba_status st = enter(h, stream);
  if (st != BA_OK) return st;
  if (!mask) {
    h->fixed = nullptr;  // the allocation (if any) stays owned by the problem
  } else {
    if (!h->fixed_buf) CU(h->alloc(&h->fixed_buf, 9ull * h->C));
    CU(cudaMemcpyAsync(h->fixed_buf, mask, 9ull * h->C, cudaMemcpyDefault, h->s));
    h->fixed = h->fixed_buf;
  }
  if (h->gexec) {
    // the captured trial bakes in the mask pointer: capture again on next use
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  return leave(h, stream);
}

ba_status ba_backward(ba_problem* h, double lambda, int maxiter, double tol, const void* dL_dcams,
                      const void* dL_dpoints, void* dL_dpixels_out, void* dL_dcams0_out, void* dL_dpoints0_out,
                      int* iters, double* rel_res, void* stream) {
  if (!h || !dL_dpixels_out) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  if (maxiter < 0 || maxiter > 100000 || !(tol >= 0) || !(lambda >= 0))
    return fail(BA_ERR_INVALID_ARG, "bad lambda/maxiter/tol");
  if (h->prec == BA_PREC_F32)
    return backward_via_f64(h, lambda, maxiter, tol, (const float*)dL_dcams, (const float*)dL_dpoints,
                            (float*)dL_dpixels_out, (float*)dL_dcams0_out, (float*)dL_dpoints0_out, iters, rel_res,
                            stream);
  ba_status st = enter(h, stream);
  if (st != BA_OK) return st;
  st = set_probe_lambda(h, lambda);
  if (st != BA_OK) return st;
  st = set_flag(h, offsetof(DevState, need_lin), 1);
  if (st != BA_OK) return st;
  const double* lp = &h->st->lam_probe;
  BA_DISPATCH(h, enqueue_backward, lp, maxiter, tol, dL_dcams, dL_dpoints, dL_dpixels_out, dL_dcams0_out,
              dL_dpoints0_out);
  if (dL_dpoints0_out) CU(cudaMemsetAsync(dL_dpoints0_out, 0, 3ull * h->P * h->tsize, h->s));
  CU(cudaGetLastError());
  // the gradient slots now hold the adjoint right-hand side: linearise again
  // before the next trial
  st = set_flag(h, offsetof(DevState, need_lin), 1);
  if (st != BA_OK) return st;
  if (iters || rel_res) {
    DevState ds;
    CU(cudaMemcpyAsync(&ds, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->s));
    CU(cudaStreamSynchronize(h->s));
    if (iters) *iters = ds.pcg_iters;
    if (rel_res) *rel_res = ds.pcg_rel;
  }
  return leave(h, stream);
}

ba_status ba_set_preconditioner(ba_problem* h, const float* params, void* stream) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "NULL problem");
  ba_status st = enter(h, stream);
  if (st != BA_OK) return st;
  if (params) {
    st = ensure_learn_buffers(h);
    if (st != BA_OK) return st;
    CU(cudaMemcpyAsync(h->mlp, params, (size_t)MLP_NPARAM * 4, cudaMemcpyDefault, h->s));
  }
  if (h->learned != (params != nullptr) && h->gexec) {
    // the captured trial has the other preconditioner: capture again
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  h->learned = params != nullptr;
  return leave(h, stream);
}

ba_status ba_learn_collect(ba_problem* h, double lambda, int K, const float* zhat, float* X_out, float* Ahat_out,
                           float* Yhat_out, double* D_out, void* stream) {
  if (!h || !X_out || !Ahat_out || (K > 0 && (!zhat || !Yhat_out)))
    return fail(BA_ERR_INVALID_ARG, "NULL argument");
  if (K < 0 || K > MLP_KMAX || !(lambda > 0)) return fail(BA_ERR_INVALID_ARG, "need 0 <= K <= %d, lambda > 0", MLP_KMAX);
  ba_status st = enter(h, stream);
  if (st != BA_OK) return st;
  st = ensure_learn_buffers(h);
  if (st != BA_OK) return st;
  st = set_probe_lambda(h, lambda);
  if (st != BA_OK) return st;
  st = set_flag(h, offsetof(DevState, need_lin), 1);
  if (st != BA_OK) return st;
  BA_DISPATCH(h, enqueue_collect, &h->st->lam_probe, K, zhat, X_out, Ahat_out, Yhat_out);
  CU(cudaGetLastError());
  if (D_out) CU(cudaMemcpyAsync(D_out, h->Dsc, 72ull * h->C, cudaMemcpyDeviceToDevice, h->s));
  return leave(h, stream);
}

ba_status ba_learn_slow_probes(ba_problem* h, double lambda, int n, const int* iters, int maxiter_ref,
                               double tol_ref, float* zhat_out, void* stream) {
  if (!h || (n > 0 && (!iters || !zhat_out))) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  if (n < 0 || n > MLP_KMAX || !(lambda > 0) || maxiter_ref < 1 || maxiter_ref > 100000 || !(tol_ref >= 0))
    return fail(BA_ERR_INVALID_ARG, "need 0 <= n <= %d, lambda > 0, 1 <= maxiter_ref <= 100000", MLP_KMAX);
  for (int j = 0; j < n; ++j)
    if (iters[j] < 0 || iters[j] > 100000) return fail(BA_ERR_INVALID_ARG, "iters out of range");
  if (n == 0) return BA_OK;
  ba_status st = enter(h, stream);
  if (st != BA_OK) return st;
  st = ensure_learn_buffers(h);
  if (st != BA_OK) return st;
  double* xref = nullptr;
  CU(cudaMalloc(&xref, 72ull * h->C));
  st = set_probe_lambda(h, lambda);
  if (st == BA_OK) st = set_flag(h, offsetof(DevState, need_lin), 1);
  if (st == BA_OK) {
    BA_DISPATCH(h, enqueue_slow_probes, &h->st->lam_probe, n, iters, maxiter_ref, tol_ref, zhat_out, xref);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) st = fail(BA_ERR_CUDA, "slow probes failed: %s", cudaGetErrorString(e));
  }
  cudaFree(xref);
  if (st != BA_OK) return st;
  return leave(h, stream);
}

uint64_t ba_kernel_launch_count(void) { return ba::g_launches.load(); }

ba_status ba_set_exchange(ba_problem* h, ba_exchange_fn fn, void* ctx, double* xbuf, size_t cap) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "NULL problem");
  if (fn && (!xbuf || cap < BA_EXCHANGE_CAP(h->C)))
    return fail(BA_ERR_INVALID_ARG, "the exchange buffer must hold BA_EXCHANGE_CAP(C) = %zu doubles",
                (size_t)BA_EXCHANGE_CAP(h->C));
  if (fn && (h->learned || h->opt.solver != BA_SOLVER_PCG))
    return fail(BA_ERR_INVALID_ARG, "a partitioned problem uses block-Jacobi PCG");
  if (fn && !h->ident_ptr) {
    std::vector<int32_t> id(h->C + 1);
    for (int c = 0; c <= h->C; ++c) id[c] = c;
    CU(h->alloc(&h->ident_ptr, (h->C + 1) * 4));
    CU(cudaMemcpy(h->ident_ptr, id.data(), (h->C + 1) * 4, cudaMemcpyHostToDevice));
    CU(h->alloc(&h->camsum, (size_t)PART * h->C * 8));
    CU(h->alloc(&h->U_loc, 45ull * h->C * 8));
    CU(h->alloc(&h->gc_loc, 9ull * h->C * 8));
    CU(h->alloc(&h->xscal, 8 * 8));
  }
  CU(cudaStreamSynchronize(h->s));
  h->xch = fn;
  h->xctx = ctx;
  h->xbuf = xbuf;
  h->xcap = fn ? cap : 0;
  h->xerr = 0;
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  // the cost is a sum over the parts now (or this problem's alone again);
  // the linearisation's sums too
  ba_status st = set_flag(h, offsetof(DevState, need_cost), 1);
  if (st == BA_OK) st = set_flag(h, offsetof(DevState, need_lin), 1);
  if (st == BA_OK) CU(cudaStreamSynchronize(h->s));
  return st;
}

ba_status ba_get_layout(const ba_problem* h, int64_t* out, int n) {
  if (!h || !out || n < 0) return fail(BA_ERR_INVALID_ARG, "bad argument");
  const int64_t v[BA_LAYOUT_COUNT] = {h->npieces, h->nchunks, h->fa ? 1 : 0, h->mf ? 0 : 1};
  for (int i = 0; i < n; ++i) out[i] = i < BA_LAYOUT_COUNT ? v[i] : 0;
  return BA_OK;
}

ba_status ba_profile_trials(ba_problem* h, int iters, ba_kernel_times* out) {
  if (!h || !out || iters < 0) return fail(BA_ERR_INVALID_ARG, "bad argument");
  memset(out, 0, sizeof(*out));
  DevState ds;
  CU(cudaMemcpyAsync(&ds, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->s));
  CU(cudaStreamSynchronize(h->s));
  const long long t0 = ds.trials;
  const int lin0 = ds.need_lin;
  std::vector<ba_problem::ProfRec> recs;
  cudaEvent_t ea, eb;
  CU(cudaEventCreate(&ea));
  CU(cudaEventCreate(&eb));
  h->prof = &recs;
  CU(cudaEventRecord(ea, h->s));
  for (int i = 0; i < iters; ++i) {
    h->prof_trial = i;
    enqueue_trial_any(h);
  }
  CU(cudaEventRecord(eb, h->s));
  h->prof = nullptr;
  cudaError_t e = cudaStreamSynchronize(h->s);
  std::vector<ba_iter_stats> st(iters);
  for (int i = 0; i < iters && e == cudaSuccess; ++i)
    e = cudaMemcpy(&st[i], h->stats + ((t0 + i) % h->cap), sizeof(ba_iter_stats), cudaMemcpyDeviceToHost);
  float tm = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&tm, ea, eb);
  out->trial_ms = tm;
  for (auto& r : recs) {
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    const bool lin = r.trial == 0 ? lin0 != 0 : st[r.trial - 1].accepted != 0;
    bool did = true;
    if (r.k == -2) did = lin;                          // gated linearisation kernels
    else if (r.k >= 0) did = r.k < st[r.trial].pcg_iters;  // PCG launches after convergence exit at once
    if (did) {
      out->ms[r.kind] += ms;
      out->launches[r.kind] += 1;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  cudaEventDestroy(ea);
  cudaEventDestroy(eb);
  if (e != cudaSuccess) return fail(BA_ERR_CUDA, "profiling failed: %s", cudaGetErrorString(e));
  return BA_OK;
}

}  // extern "C"
