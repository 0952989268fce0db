// The problem object behind the C ABI (shared by the library's translation
// units; not part of the public interface).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "ba.h"
#include "ba_kernels.cuh"

struct ba_problem {
  int C = 0, P = 0, O = 0, prec = 0;
  bool mf = false;  // recompute the Jacobian factors in every pass
  size_t tsize = 8;
  ba_options opt{};
  cudaStream_t s = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<void*> allocs;
  // structure (symbolic phase)
  // Points are renumbered internally (sorted by the first camera that sees
  // them) so that the points of one camera are close together in memory.
  // pt_idx, perm_*, rowptr_pt and every per-point array use the internal
  // numbering; pnew[new] = caller's index, pnewpos[caller's] = new.
  int32_t *cam_idx = nullptr, *pt_idx = nullptr;
  int32_t *perm_cam = nullptr, *rowptr_cam = nullptr, *perm_pt = nullptr, *rowptr_pt = nullptr;
  int32_t *pnew = nullptr, *pnewpos = nullptr;
  // the symbolic phase in the caller's numbering (ba_get_csr)
  int32_t *xperm_cam = nullptr, *xperm_pt = nullptr, *xrowptr_pt = nullptr;
  void* pts_tmp = nullptr;  // [P][3] staging for reordering parameters
  void* cams_tmp = nullptr;  // [C][9] staging for parameters in and out
  bool cost_pending = false;  // DevState::need_cost set and not yet evaluated
  uint8_t* fixed = nullptr;  // [C][9] frozen camera parameters, or NULL
  uint8_t* fixed_buf = nullptr;
  int32_t *cm_pt = nullptr, *pm_cam = nullptr, *pm_pt = nullptr;
  int32_t* pm2cm = nullptr;  // camera-major slot of each point-major slot
  int nchunks = 0;
  int32_t* pchunk = nullptr;  // [nchunks + 1] first point of each point chunk
  // fused point-major pass A (recompute mode): the distinct cameras of each
  // point chunk (chunk_cams[chunk_cam_ptr[k] ..]) and each point-major slot's
  // position in its chunk's list
  bool fa = false;
  int fa_nc = 0;  // the most cameras one point chunk sees (fused pass A)
  int32_t *chunk_cams = nullptr, *chunk_cam_ptr = nullptr;
  int16_t* pm_lc = nullptr;
  int4* chunk_hdr = nullptr;  // [nchunks][2] headers of the fused pass
  void *cm_px = nullptr, *pm_px = nullptr, *px_in = nullptr;
  int npieces = 0;
  int32_t *piece_cam = nullptr, *piece_beg = nullptr, *piece_end = nullptr, *cam_piece_ptr = nullptr;
  // parameters, double-buffered (current / trial)
  void *cams = nullptr, *pts = nullptr;
  // linearisation
  void *camtab = nullptr, *Jcm = nullptr;
  void* Jpm = nullptr;  // stored mode: the planes in point-major order (fused pass A)
  void *ptab = nullptr;  // [P][8]: X, 0, t, 0
  void *zbuf = nullptr;  // [O][4]: pass A1 output, camera-major
  void *cm_sw = nullptr, *pm_sw = nullptr;  // sqrt(w) per observation (recompute mode, robust loss)
  double *U = nullptr, *gc = nullptr, *V = nullptr, *gp = nullptr;
  void *Vinv = nullptr, *y0 = nullptr;
  // PCG
  double *Minv = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  void *pT = nullptr, *xT = nullptr, *dp = nullptr;
  double* part = nullptr;
  int ncb = 0, npb = 0;
  double *dot_pq = nullptr, *dot_rz = nullptr, *dot_rr = nullptr, *dot_bb = nullptr;
  double *dot_gc = nullptr, *dot_gp = nullptr;
  // learned block-Jacobi correction (ba_set_preconditioner, ba_learn_collect)
  bool learned = false;
  float* mlp = nullptr;     // [13293] network parameters
  double* Sii = nullptr;    // [C][45] diagonal blocks of S (packed upper)
  float* Xf = nullptr;      // [C][96] features
  float* Ef = nullptr;      // [C][45] network output
  double* Dsc = nullptr;    // [C][9] scales diag(S_ii)
  double* kap = nullptr;    // [C] coupling sums of the probes (feature 93)
  // direct solver (BA_SOLVER_CHOLESKY): nseg partial copies of S, the band
  // tiles of S (then L; the band is the whole lower triangle), 1 / L_cc,
  // L_JJ^{-T}, the work vector, the factorisation's flags (tile final and
  // tile updates [bnb bnb] each, counters [5], failure [1], inverse final
  // [bnb]) and its task list
  double* Wd = nullptr;     // [O][27] W = Jc^T Jp per observation
  double* Spart = nullptr;
  int nseg = 1;
  double *bT = nullptr, *brs = nullptr, *bUi = nullptr, *dy = nullptr;
  int* bflag = nullptr;
  int4* btask = nullptr;
  int bnb = 0, bwt = 0, bntask = 0, bncrit = 0, band_grid = 0, band_crit = 0;
  size_t bT_bytes = 0, bflag_count = 0;
  ba::DevState* st = nullptr;
  ba_iter_stats* stats = nullptr;
  int cap = 0;
  // graph of one trial
  cudaGraphExec_t gexec = nullptr;
  size_t gnodes = 0;
  // per-launch CUDA events (ba_profile_trials only)
  struct ProfRec {
    int kind, trial, k;
    cudaEvent_t a, b;
  };
  std::vector<ProfRec>* prof = nullptr;
  int prof_trial = 0;

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
  // FP32 problems: an FP64 copy for the adjoint solve (ba_backward)
  ba_problem* twin = nullptr;
  // point-partitioned problem (ba_set_exchange): the caller's all-reduce and
  // its device buffer; identity piece pointers and the per-camera /
  // scalar partials exchanged; the first exchange error of a trial
  ba_exchange_fn xch = nullptr;
  void* xctx = nullptr;
  double* xbuf = nullptr;
  size_t xcap = 0;
  int32_t* ident_ptr = nullptr;  // [C+1] = 0..C: one summed row per camera
  double* camsum = nullptr;      // [C][PART] Schur-pass sums; [C][9] pass-B sums
  double* U_loc = nullptr;       // [C][45] this part's U, [C][9] its gc
  double* gc_loc = nullptr;
  double* xscal = nullptr;       // [8] trial and cost sums
  int xerr = 0;
  ~ba_problem() {
    if (twin) ba_problem_destroy(twin);
    if (gexec) cudaGraphExecDestroy(gexec);
    for (void* v : allocs) cudaFree(v);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (s) cudaStreamDestroy(s);
  }
};

