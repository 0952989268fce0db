// Learned block-Jacobi correction: per-camera features of the reduced camera
// system, a 96-64-64-45 ReLU network on the tensor cores (BF16 operands,
// FP32 accumulation) for inference and training, and the SPD preconditioner
// block built from its output.  Not in the paper (its PCG uses a diagonal
// preconditioner, Sec. IV-C); the block it corrects is the 9x9 block-Jacobi
// inverse of the plain method.
//
//   scaled coordinates  D = diag(S_ii), S^ = D^{-1/2} S D^{-1/2}
//   features x_i (96)   36 off-diagonal entries of S^_ii; 45 entries of the
//                       scaled point-elimination term R^ = D^{-1/2}(U*_i -
//                       S_ii)D^{-1/2}, each divided by sqrt((1+R^_aa)(1+R^_bb));
//                       (ln D_a - mean ln D) / 10; log10(lambda) / 8;
//                       log10(1 + observations) / 4; 1; zeros
//   network             h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2),
//                       e = W3 h2 + b3; flat parameters W1 [64][96], b1,
//                       W2 [64][64], b2, W3 [45][64], b3 (13293 floats)
//   block               G lower triangular, G_ab = e_{a(a+1)/2+b} (a > b),
//                       G_aa = exp(e_{a(a+1)/2+a});  M_i = L^{-T} G G^T L^{-1},
//                       L = chol(S_ii): SPD for any e, e = 0 gives S_ii^{-1}
//   training loss       mean over cameras of 1/(9K) sum_k |M^_i y^_ik - z^_ik|^2,
//                       M^_i = A^T G G^T A, A = chol(S^_ii)^{-1}, y^ = S^ z^
//                       for Rademacher probes z^ (E_z |M S z - z|^2 in the
//                       scaled coordinates, separable per camera)
#pragma once

#include <cuda_bf16.h>

#include "ba_kernels.cuh"

namespace ba {

constexpr int MLP_FIN = 96, MLP_H = 64, MLP_FOUT = 45, MLP_FOUTP = 48;
constexpr int MLP_OW1 = 0;
constexpr int MLP_OB1 = MLP_OW1 + MLP_H * MLP_FIN;
constexpr int MLP_OW2 = MLP_OB1 + MLP_H;
constexpr int MLP_OB2 = MLP_OW2 + MLP_H * MLP_H;
constexpr int MLP_OW3 = MLP_OB2 + MLP_H;
constexpr int MLP_OB3 = MLP_OW3 + MLP_FOUT * MLP_H;
constexpr int MLP_NPARAM = MLP_OB3 + MLP_FOUT;
static_assert(MLP_NPARAM == 13293, "parameter layout");
constexpr int MLP_ROWS = 64;     // samples per CTA tile (16 per warp)
constexpr int MLP_THREADS = 128;
constexpr int MLP_KMAX = 16;     // probes per sample

__device__ __forceinline__ int tri_lo(int a, int b) { return a * (a + 1) / 2 + b; }

// ---------------------------------------------------------------------------
// Features (one thread per camera, FP64)
// ---------------------------------------------------------------------------

// Cholesky of the scaled block in W (lower, row-major 9x9) and its inverse
// (lower) in Ai; false if not positive definite.
__device__ inline bool chol_inv9(const double* __restrict__ A, double* __restrict__ L, double* __restrict__ Li) {
#pragma unroll 1
  for (int j = 0; j < 9; ++j) {
    double d = A[9 * j + j];
#pragma unroll 1
    for (int k = 0; k < j; ++k) d -= L[9 * j + k] * L[9 * j + k];
    if (!(d > 0.0) || !isfinite(d)) return false;
    const double ljj = sqrt(d);
    L[9 * j + j] = ljj;
#pragma unroll 1
    for (int i = j + 1; i < 9; ++i) {
      double s = A[9 * i + j];
#pragma unroll 1
      for (int k = 0; k < j; ++k) s -= L[9 * i + k] * L[9 * j + k];
      L[9 * i + j] = s / ljj;
    }
  }
#pragma unroll 1
  for (int i = 0; i < 9; ++i) {
#pragma unroll 1
    for (int j = 0; j < 9; ++j) Li[9 * i + j] = 0.0;
    Li[9 * i + i] = 1.0 / L[9 * i + i];
#pragma unroll 1
    for (int j = 0; j < i; ++j) {
      double s = 0.0;
#pragma unroll 1
      for (int k = j; k < i; ++k) s += L[9 * i + k] * Li[9 * k + j];
      Li[9 * i + j] = -s * Li[9 * i + i];
    }
  }
  return true;
}

// probes of the coupling feature (k_coup_probe_in, k_coup_acc)
constexpr int COUPLING_PROBES = 2;

// Features x (FP32 [C][96]) and, when Ahat is given, A = chol(S^_ii)^{-1}
// (FP32 [C][45], packed lower row-major) and D (double [C][9]).  Sii and U
// are packed upper triangles [C][45]; lam the damping of U*; kap the
// coupling sums of k_coup_acc (NULL: coupling 0).  A camera whose S_ii is
// not positive definite gets x = 0, A = 0, D = 0.
static __global__ void __launch_bounds__(CAM_THREADS)
k_learn_features(int C, const double* __restrict__ Sii, const double* __restrict__ U,
                 const double* __restrict__ lam_ptr, double dmin, double dmax,
                 const int32_t* __restrict__ rowptr_cam, float* __restrict__ X, float* __restrict__ Ahat,
                 double* __restrict__ Dout, const double* __restrict__ kap) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const double lam = *lam_ptr;
  const double* S = Sii + 45LL * c;
  const double* Uc = U + 45LL * c;
  float* x = X + (long long)MLP_FIN * c;
  double d[9], s[9];
  bool ok = true;
  for (int a = 0; a < 9; ++a) {
    d[a] = S[sym9(a, a)];
    ok = ok && d[a] > 0.0 && isfinite(d[a]);
    s[a] = ok ? 1.0 / sqrt(d[a]) : 0.0;
  }
  double Sh[81], L[81], Li[81];
  if (ok) {
    for (int a = 0; a < 9; ++a)
      for (int b = 0; b < 9; ++b) Sh[9 * a + b] = S[sym9_rt(a, b)] * s[a] * s[b];
    ok = chol_inv9(Sh, L, Li);
  }
  if (!ok) {
    for (int i = 0; i < MLP_FIN; ++i) x[i] = 0.f;
    if (Ahat)
      for (int i = 0; i < 45; ++i) Ahat[45LL * c + i] = 0.f;
    if (Dout)
      for (int i = 0; i < 9; ++i) Dout[9LL * c + i] = 0.0;
    return;
  }
  int f = 0;
  for (int a = 0; a < 9; ++a)
    for (int b = a + 1; b < 9; ++b) x[f++] = (float)Sh[9 * a + b];
  double rd[9];
  for (int a = 0; a < 9; ++a) {
    const double us = Uc[sym9(a, a)] + damp(Uc[sym9(a, a)], lam, dmin, dmax);
    rd[a] = (us - d[a]) * s[a] * s[a];
  }
  for (int a = 0; a < 9; ++a)
    for (int b = a; b < 9; ++b) {
      const double us = Uc[sym9(a, b)] + (a == b ? damp(Uc[sym9(a, a)], lam, dmin, dmax) : 0.0);
      const double r = (us - S[sym9(a, b)]) * s[a] * s[b];
      x[f++] = (float)(r / sqrt((1.0 + rd[a]) * (1.0 + rd[b])));
    }
  double mean = 0.0;
  for (int a = 0; a < 9; ++a) mean += log(d[a]);
  mean /= 9.0;
  for (int a = 0; a < 9; ++a) x[f++] = (float)((log(d[a]) - mean) / 10.0);
  x[f++] = (float)(log10(lam) / 8.0);
  x[f++] = (float)(log10(1.0 + (double)(rowptr_cam[c + 1] - rowptr_cam[c])) / 4.0);
  x[f++] = 1.f;
  x[f++] = kap ? (float)(log10(1.0 + sqrt(kap[c] / COUPLING_PROBES)) / 4.0) : 0.f;
  while (f < MLP_FIN) x[f++] = 0.f;
  if (Ahat)
    for (int a = 0; a < 9; ++a)
      for (int b = 0; b <= a; ++b) Ahat[45LL * c + tri_lo(a, b)] = (float)Li[9 * a + b];
  if (Dout)
    for (int a = 0; a < 9; ++a) Dout[9LL * c + a] = d[a];
}

// ---------------------------------------------------------------------------
// The network on the tensor cores
// ---------------------------------------------------------------------------

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}
__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) {  // p[0], p[1]; 4-byte aligned
  return *reinterpret_cast<const uint32_t*>(p);
}

// C[16 x 8*NT] += A[16 x 16*KS] B, A row-major bf16 at a (row stride lda),
// B given as Bt [n][k] row-major bf16 at bt (row stride ldb) -- the
// "col-major B" of mma.sync.  One warp; acc in the C-fragment layout.
template <int KS, int NT>
__device__ __forceinline__ void warp_gemm_rowA(const __nv_bfloat16* __restrict__ a, int lda,
                                               const __nv_bfloat16* __restrict__ bt, int ldb, float (&acc)[NT][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
    const int k0 = 16 * ks + 2 * t;
    uint32_t af[4];
    af[0] = ld_pair(a + g * lda + k0);
    af[1] = ld_pair(a + (g + 8) * lda + k0);
    af[2] = ld_pair(a + g * lda + k0 + 8);
    af[3] = ld_pair(a + (g + 8) * lda + k0 + 8);
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      uint32_t bf[2];
      bf[0] = ld_pair(bt + (8 * nt + g) * ldb + k0);
      bf[1] = ld_pair(bt + (8 * nt + g) * ldb + k0 + 8);
      mma_bf16_16816(acc[nt], af, bf);
    }
  }
}

// One 16x8 tile of C = P^T Q summed over the 64 rows of a CTA tile: P [64][ldp]
// and Q [64][ldq] row-major bf16; the tile covers C rows m0..m0+15 (columns of
// P) and C columns n0..n0+7 (columns of Q).
__device__ __forceinline__ void warp_gemm_tn_tile(const __nv_bfloat16* __restrict__ P, int ldp, int m0,
                                                  const __nv_bfloat16* __restrict__ Q, int ldq, int n0,
                                                  float (&acc)[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int ks = 0; ks < MLP_ROWS / 16; ++ks) {
    const int r0 = 16 * ks + 2 * t;
    uint32_t af[4], bf[2];
    af[0] = pack_bf16(P[r0 * ldp + m0 + g], P[(r0 + 1) * ldp + m0 + g]);
    af[1] = pack_bf16(P[r0 * ldp + m0 + g + 8], P[(r0 + 1) * ldp + m0 + g + 8]);
    af[2] = pack_bf16(P[(r0 + 8) * ldp + m0 + g], P[(r0 + 9) * ldp + m0 + g]);
    af[3] = pack_bf16(P[(r0 + 8) * ldp + m0 + g + 8], P[(r0 + 9) * ldp + m0 + g + 8]);
    bf[0] = pack_bf16(Q[r0 * ldq + n0 + g], Q[(r0 + 1) * ldq + n0 + g]);
    bf[1] = pack_bf16(Q[(r0 + 8) * ldq + n0 + g], Q[(r0 + 9) * ldq + n0 + g]);
    mma_bf16_16816(acc, af, bf);
  }
}

// Shared memory of the network kernels: the forward part first (the
// inference kernel allocates only up to `dE`), then what training adds.
struct MlpSmem {
  __nv_bfloat16 W1[MLP_H][MLP_FIN];     // [out][in]: B operand of layer 1
  __nv_bfloat16 W2[MLP_H][MLP_H];
  __nv_bfloat16 W3[MLP_FOUTP][MLP_H];
  float b1[MLP_H], b2[MLP_H], b3[MLP_FOUTP];
  __nv_bfloat16 X[MLP_ROWS][MLP_FIN];
  __nv_bfloat16 H1[MLP_ROWS][MLP_H];
  __nv_bfloat16 H2[MLP_ROWS][MLP_H];
  float E[MLP_ROWS][MLP_FOUTP];         // network output, then dl/de (FP32)
  // training only
  __nv_bfloat16 dE[MLP_ROWS][MLP_FOUTP];
  __nv_bfloat16 W2T[MLP_H][MLP_H];      // [in][out]: B operand of dh1 = dh2 W2
  __nv_bfloat16 W3T[MLP_H][MLP_FOUTP];  // [in][out]: B operand of dh2 = de W3
  __nv_bfloat16 dH2[MLP_ROWS][MLP_H];
  __nv_bfloat16 dH1[MLP_ROWS][MLP_H];
  float dH2f[MLP_ROWS][MLP_H];
  float dH1f[MLP_ROWS][MLP_H];
  float gW1[MLP_H][MLP_FIN];
  float gW2[MLP_H][MLP_H];
  float gW3[MLP_FOUTP][MLP_H];
  float gb1[MLP_H], gb2[MLP_H], gb3[MLP_FOUTP];
  double rowloss[MLP_ROWS];
};
constexpr size_t MLP_SMEM_FWD = offsetof(MlpSmem, dE);
constexpr size_t MLP_SMEM_TRAIN = sizeof(MlpSmem);

// Stage the FP32 parameters as BF16 operands (and transposes) and FP32 biases.
__device__ inline void mlp_stage_weights(const float* __restrict__ p, MlpSmem& S, bool train) {
  for (int i = threadIdx.x; i < MLP_H * MLP_FIN; i += blockDim.x)
    S.W1[i / MLP_FIN][i % MLP_FIN] = __float2bfloat16_rn(p[MLP_OW1 + i]);
  for (int i = threadIdx.x; i < MLP_H * MLP_H; i += blockDim.x) {
    const __nv_bfloat16 w = __float2bfloat16_rn(p[MLP_OW2 + i]);
    S.W2[i / MLP_H][i % MLP_H] = w;
    if (train) S.W2T[i % MLP_H][i / MLP_H] = w;
  }
  for (int i = threadIdx.x; i < MLP_FOUTP * MLP_H; i += blockDim.x) {
    const int o = i / MLP_H, k = i % MLP_H;
    const __nv_bfloat16 w = __float2bfloat16_rn(o < MLP_FOUT ? p[MLP_OW3 + o * MLP_H + k] : 0.f);
    S.W3[o][k] = w;
    if (train) S.W3T[k][o] = w;
  }
  for (int i = threadIdx.x; i < MLP_H; i += blockDim.x) {
    S.b1[i] = p[MLP_OB1 + i];
    S.b2[i] = p[MLP_OB2 + i];
  }
  for (int i = threadIdx.x; i < MLP_FOUTP; i += blockDim.x) S.b3[i] = i < MLP_FOUT ? p[MLP_OB3 + i] : 0.f;
}

// Forward pass of the 64 rows of one tile (X already staged): each warp its
// 16 rows; leaves H1, H2 (BF16, after ReLU) and E (FP32) in shared memory.
__device__ inline void mlp_tile_forward(MlpSmem& S) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = 16 * warp;
  {
    float acc[8][4] = {};
    warp_gemm_rowA<MLP_FIN / 16, 8>(&S.X[r0][0], MLP_FIN, &S.W1[0][0], MLP_FIN, acc);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int col = 8 * nt + 2 * t + q;
          S.H1[r0 + g + 8 * h][col] = __float2bfloat16_rn(fmaxf(acc[nt][2 * h + q] + S.b1[col], 0.f));
        }
  }
  __syncwarp();
  {
    float acc[8][4] = {};
    warp_gemm_rowA<MLP_H / 16, 8>(&S.H1[r0][0], MLP_H, &S.W2[0][0], MLP_H, acc);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int col = 8 * nt + 2 * t + q;
          S.H2[r0 + g + 8 * h][col] = __float2bfloat16_rn(fmaxf(acc[nt][2 * h + q] + S.b2[col], 0.f));
        }
  }
  __syncwarp();
  {
    float acc[6][4] = {};
    warp_gemm_rowA<MLP_H / 16, 6>(&S.H2[r0][0], MLP_H, &S.W3[0][0], MLP_H, acc);
#pragma unroll
    for (int nt = 0; nt < 6; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int col = 8 * nt + 2 * t + q;
          S.E[r0 + g + 8 * h][col] = acc[nt][2 * h + q] + S.b3[col];
        }
  }
  __syncwarp();
}

__device__ inline void mlp_stage_x(const float* __restrict__ X, int n, int row0, MlpSmem& S) {
  for (int i = threadIdx.x; i < MLP_ROWS * MLP_FIN; i += blockDim.x) {
    const int r = i / MLP_FIN, k = i % MLP_FIN;
    const int row = row0 + r;
    S.X[r][k] = __float2bfloat16_rn(row < n ? X[(long long)row * MLP_FIN + k] : 0.f);
  }
}

// Inference: E_out [n][45] (FP32) = network(X [n][96]).  One tile per CTA.
static __global__ void __launch_bounds__(MLP_THREADS)
k_mlp_forward(int n, const float* __restrict__ params, const float* __restrict__ X, float* __restrict__ E_out) {
  extern __shared__ __align__(16) unsigned char mlp_raw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(mlp_raw);
  const int row0 = blockIdx.x * MLP_ROWS;
  mlp_stage_weights(params, S, false);
  mlp_stage_x(X, n, row0, S);
  __syncthreads();
  mlp_tile_forward(S);
  __syncthreads();
  for (int i = threadIdx.x; i < MLP_ROWS * MLP_FOUT; i += blockDim.x) {
    const int r = i / MLP_FOUT, c = i % MLP_FOUT;
    if (row0 + r < n) E_out[(long long)(row0 + r) * MLP_FOUT + c] = S.E[r][c];
  }
}

// Per-sample probe loss and dl/de (FP32), one lane per sample: e from S.E
// row r; writes dl/de (scaled by `scale` = 1 / (9 K n)) back to S.E row r
// and returns the sample's loss 1/(9K) sum_k |M^ y^_k - z^_k|^2.
__device__ inline double probe_row(float* __restrict__ e, const float* __restrict__ Ah, const float* __restrict__ Y,
                                   const float* __restrict__ Z, int K, float scale) {
  float G[45], A[45], dG[45];
#pragma unroll
  for (int a = 0; a < 9; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      const int i = tri_lo(a, b);
      G[i] = a == b ? expf(e[i]) : e[i];
      A[i] = Ah[i];
      dG[i] = 0.f;
    }
  double loss = 0.0;
  for (int k = 0; k < K; ++k) {
    float y[9], z[9], u[9], v[9], w[9], dm[9], dw[9], dv[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      y[a] = Y[9 * k + a];
      z[a] = Z[9 * k + a];
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) {  // u = A y
      float s = 0.f;
#pragma unroll
      for (int b = 0; b <= a; ++b) s += A[tri_lo(a, b)] * y[b];
      u[a] = s;
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) {  // v = G^T u
      float s = 0.f;
#pragma unroll
      for (int a = c; a < 9; ++a) s += G[tri_lo(a, c)] * u[a];
      v[c] = s;
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) {  // w = G v
      float s = 0.f;
#pragma unroll
      for (int c = 0; c <= a; ++c) s += G[tri_lo(a, c)] * v[c];
      w[a] = s;
    }
    float rr = 0.f;
#pragma unroll
    for (int b = 0; b < 9; ++b) {  // m = A^T w, r = m - z
      float s = 0.f;
#pragma unroll
      for (int a = b; a < 9; ++a) s += A[tri_lo(a, b)] * w[a];
      const float r = s - z[b];
      rr += r * r;
      dm[b] = 2.f * scale * r;
    }
    loss += (double)rr;
#pragma unroll
    for (int a = 0; a < 9; ++a) {  // dw = A dm
      float s = 0.f;
#pragma unroll
      for (int b = 0; b <= a; ++b) s += A[tri_lo(a, b)] * dm[b];
      dw[a] = s;
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) {  // dv = G^T dw
      float s = 0.f;
#pragma unroll
      for (int a = c; a < 9; ++a) s += G[tri_lo(a, c)] * dw[a];
      dv[c] = s;
    }
#pragma unroll
    for (int a = 0; a < 9; ++a)
#pragma unroll
      for (int c = 0; c <= a; ++c) dG[tri_lo(a, c)] += dw[a] * v[c] + u[a] * dv[c];
  }
#pragma unroll
  for (int a = 0; a < 9; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      const int i = tri_lo(a, b);
      e[i] = a == b ? dG[i] * G[i] : dG[i];
    }
  return loss / (9.0 * K);
}

// Training: forward, probe loss, backward over the rows [0, n) in tiles of
// 64 (tile t handled by CTA t % gridDim.x, in order); per-CTA gradient sums
// (FP32, layout of the parameters) in grad_part [gridDim.x][13293] and loss
// sums in loss_part [gridDim.x].  dl/de carries 1 / (9 K n).
static __global__ void __launch_bounds__(MLP_THREADS)
k_mlp_train(int n, int K, const float* __restrict__ params, const float* __restrict__ X,
            const float* __restrict__ Ahat, const float* __restrict__ Yhat, const float* __restrict__ Zhat,
            float* __restrict__ grad_part, double* __restrict__ loss_part) {
  extern __shared__ __align__(16) unsigned char mlp_raw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(mlp_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  mlp_stage_weights(params, S, true);
  for (int i = tid; i < MLP_H * MLP_FIN; i += blockDim.x) (&S.gW1[0][0])[i] = 0.f;
  for (int i = tid; i < MLP_H * MLP_H; i += blockDim.x) (&S.gW2[0][0])[i] = 0.f;
  for (int i = tid; i < MLP_FOUTP * MLP_H; i += blockDim.x) (&S.gW3[0][0])[i] = 0.f;
  for (int i = tid; i < MLP_H; i += blockDim.x) S.gb1[i] = S.gb2[i] = 0.f;
  for (int i = tid; i < MLP_FOUTP; i += blockDim.x) S.gb3[i] = 0.f;
  double cta_loss = 0.0;
  const float scale = 1.f / (9.f * (float)K * (float)n);
  const int ntiles = (n + MLP_ROWS - 1) / MLP_ROWS;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int row0 = tile * MLP_ROWS;
    __syncthreads();
    mlp_stage_x(X, n, row0, S);
    __syncthreads();
    mlp_tile_forward(S);
    // probe loss and dl/de: lane r < 16 of each warp takes row 16 warp + r
    if (lane < 16) {
      const int r = 16 * warp + lane, row = row0 + r;
      double l = 0.0;
      if (row < n) {
        l = probe_row(&S.E[r][0], Ahat + 45LL * row, Yhat + 9LL * K * row, Zhat + 9LL * K * row, K, scale);
      } else {
        for (int c = 0; c < MLP_FOUTP; ++c) S.E[r][c] = 0.f;
      }
      S.rowloss[r] = l;
      for (int c = 0; c < MLP_FOUTP; ++c) S.dE[r][c] = __float2bfloat16_rn(c < MLP_FOUT ? S.E[r][c] : 0.f);
    }
    __syncwarp();
    const int r0 = 16 * warp;
    {  // dh2 = (de W3) * relu'(h2)
      float acc[8][4] = {};
      warp_gemm_rowA<MLP_FOUTP / 16, 8>(&S.dE[r0][0], MLP_FOUTP, &S.W3T[0][0], MLP_FOUTP, acc);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int row = r0 + g + 8 * h, col = 8 * nt + 2 * t + q;
            const float v = __bfloat162float(S.H2[row][col]) > 0.f ? acc[nt][2 * h + q] : 0.f;
            S.dH2f[row][col] = v;
            S.dH2[row][col] = __float2bfloat16_rn(v);
          }
    }
    __syncwarp();
    {  // dh1 = (dh2 W2) * relu'(h1)
      float acc[8][4] = {};
      warp_gemm_rowA<MLP_H / 16, 8>(&S.dH2[r0][0], MLP_H, &S.W2T[0][0], MLP_H, acc);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int row = r0 + g + 8 * h, col = 8 * nt + 2 * t + q;
            const float v = __bfloat162float(S.H1[row][col]) > 0.f ? acc[nt][2 * h + q] : 0.f;
            S.dH1f[row][col] = v;
            S.dH1[row][col] = __float2bfloat16_rn(v);
          }
    }
    __syncthreads();
    // weight gradients over the tile's 64 rows; each 16x8 output tile is
    // owned by one warp (tiles w, w+4, ...)
    for (int ot = warp; ot < 3 * 8; ot += 4) {  // gW3 [48][64] += dE^T H2
      const int m0 = 16 * (ot / 8), n0 = 8 * (ot % 8);
      float acc[4] = {};
      warp_gemm_tn_tile(&S.dE[0][0], MLP_FOUTP, m0, &S.H2[0][0], MLP_H, n0, acc);
      S.gW3[m0 + g][n0 + 2 * t] += acc[0];
      S.gW3[m0 + g][n0 + 2 * t + 1] += acc[1];
      S.gW3[m0 + g + 8][n0 + 2 * t] += acc[2];
      S.gW3[m0 + g + 8][n0 + 2 * t + 1] += acc[3];
    }
    for (int ot = warp; ot < 4 * 8; ot += 4) {  // gW2 [64][64] += dH2^T H1
      const int m0 = 16 * (ot / 8), n0 = 8 * (ot % 8);
      float acc[4] = {};
      warp_gemm_tn_tile(&S.dH2[0][0], MLP_H, m0, &S.H1[0][0], MLP_H, n0, acc);
      S.gW2[m0 + g][n0 + 2 * t] += acc[0];
      S.gW2[m0 + g][n0 + 2 * t + 1] += acc[1];
      S.gW2[m0 + g + 8][n0 + 2 * t] += acc[2];
      S.gW2[m0 + g + 8][n0 + 2 * t + 1] += acc[3];
    }
    for (int ot = warp; ot < 4 * 12; ot += 4) {  // gW1 [64][96] += dH1^T X
      const int m0 = 16 * (ot / 12), n0 = 8 * (ot % 12);
      float acc[4] = {};
      warp_gemm_tn_tile(&S.dH1[0][0], MLP_H, m0, &S.X[0][0], MLP_FIN, n0, acc);
      S.gW1[m0 + g][n0 + 2 * t] += acc[0];
      S.gW1[m0 + g][n0 + 2 * t + 1] += acc[1];
      S.gW1[m0 + g + 8][n0 + 2 * t] += acc[2];
      S.gW1[m0 + g + 8][n0 + 2 * t + 1] += acc[3];
    }
    // bias gradients: column sums of the FP32 upstream gradients, rows in order
    for (int c = tid; c < MLP_FOUTP + 2 * MLP_H; c += blockDim.x) {
      float s = 0.f;
      if (c < MLP_FOUTP) {
        for (int r = 0; r < MLP_ROWS; ++r) s += S.E[r][c];
        S.gb3[c] += s;
      } else if (c < MLP_FOUTP + MLP_H) {
        const int cc = c - MLP_FOUTP;
        for (int r = 0; r < MLP_ROWS; ++r) s += S.dH2f[r][cc];
        S.gb2[cc] += s;
      } else {
        const int cc = c - MLP_FOUTP - MLP_H;
        for (int r = 0; r < MLP_ROWS; ++r) s += S.dH1f[r][cc];
        S.gb1[cc] += s;
      }
    }
    if (tid == 0)
      for (int r = 0; r < MLP_ROWS; ++r) cta_loss += S.rowloss[r];
  }
  __syncthreads();
  float* out = grad_part + (long long)blockIdx.x * MLP_NPARAM;
  for (int i = tid; i < MLP_H * MLP_FIN; i += blockDim.x) out[MLP_OW1 + i] = (&S.gW1[0][0])[i];
  for (int i = tid; i < MLP_H; i += blockDim.x) {
    out[MLP_OB1 + i] = S.gb1[i];
    out[MLP_OB2 + i] = S.gb2[i];
  }
  for (int i = tid; i < MLP_H * MLP_H; i += blockDim.x) out[MLP_OW2 + i] = (&S.gW2[0][0])[i];
  for (int i = tid; i < MLP_FOUT * MLP_H; i += blockDim.x) out[MLP_OW3 + i] = (&S.gW3[0][0])[i];
  for (int i = tid; i < MLP_FOUT; i += blockDim.x) out[MLP_OB3 + i] = S.gb3[i];
  if (tid == 0) loss_part[blockIdx.x] = cta_loss;
}

// grad[i] = sum over the CTA partials in order (double); loss likewise
// (mean over the n samples).
static __global__ void k_mlp_reduce(int nparts, int n, const float* __restrict__ grad_part,
                             const double* __restrict__ loss_part, double* __restrict__ grad,
                             double* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < MLP_NPARAM) {
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += (double)grad_part[(long long)p * MLP_NPARAM + i];
    grad[i] = s;
  }
  if (i == 0 && loss) {
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += loss_part[p];
    *loss = s / (double)n;
  }
}

// Adam (bias-corrected) on the FP32 parameters.
static __global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const double* __restrict__ grad, int step, float lr, float b1, float b2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= MLP_NPARAM) return;
  const float gi = (float)grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.f - powf(b1, (float)step));
  const float vh = vi / (1.f - powf(b2, (float)step));
  p[i] -= lr * mh / (sqrtf(vh) + eps);
}

// ---------------------------------------------------------------------------
// The learned block in the PCG
// ---------------------------------------------------------------------------

// Per camera (after the block-Jacobi start of k_cam_combine_schur): M_i =
// L^{-T} G G^T L^{-1} from the network output e [C][45] and S_ii; if it is
// not finite the block-Jacobi inverse stays.  Then z = M r, p = z, p in the
// passes' form, and per-block partial r.z (the PCG's first r.z).
template <typename T, bool MF>
static __global__ void __launch_bounds__(CAM_THREADS)
k_learn_start(int C, const double* __restrict__ Sii, const float* __restrict__ E, const T* __restrict__ camtab,
              double* __restrict__ Minv, const double* __restrict__ r, double* __restrict__ z,
              double* __restrict__ p, T* __restrict__ pT, double* __restrict__ dot_rz1,
              const uint8_t* __restrict__ fixed, DevState* st) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double rz = 0.0;
  if (c < C) {
    double A[81], L[81], Li[81];
    const double* S = Sii + 45LL * c;
    for (int a = 0; a < 9; ++a)
      for (int b = 0; b < 9; ++b) A[9 * a + b] = S[sym9_rt(a, b)];
    double* Mc = Minv + 45LL * c;
    bool frozen = false;  // cameras with frozen parameters keep block-Jacobi
    if (fixed)
      for (int i = 0; i < 9; ++i) frozen = frozen || fixed[9LL * c + i] != 0;
    if (frozen) {
      atomicAdd(&st->fallbacks, 1);
    } else if (chol_inv9(A, L, Li)) {
      // B = G^T Li (upper x lower), M = B^T B
      double G[81];
      const float* e = E + (long long)MLP_FOUT * c;
      for (int a = 0; a < 9; ++a)
        for (int b = 0; b < 9; ++b) G[9 * a + b] = b < a ? (double)e[tri_lo(a, b)] : (a == b ? exp((double)e[tri_lo(a, a)]) : 0.0);
      double B[81];
      for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
          double s = 0.0;
          for (int d = 0; d < 9; ++d) s += G[9 * d + i] * Li[9 * d + j];
          B[9 * i + j] = s;
        }
      double M[45];
      bool fin = true;
      for (int i = 0; i < 9; ++i)
        for (int j = i; j < 9; ++j) {
          double s = 0.0;
          for (int d = 0; d < 9; ++d) s += B[9 * d + i] * B[9 * d + j];
          M[sym9(i, j)] = s;
          fin = fin && isfinite(s);
        }
      if (fin)
        for (int i = 0; i < 45; ++i) Mc[i] = M[i];
      else
        atomicAdd(&st->fallbacks, 1);
    } else {
      atomicAdd(&st->fallbacks, 1);
    }
    double rc[9], zz[9];
    for (int i = 0; i < 9; ++i) rc[i] = r[9LL * c + i];
    sym9_matvec(Mc, rc, zz);
    for (int i = 0; i < 9; ++i) {
      z[9LL * c + i] = zz[i];
      p[9LL * c + i] = zz[i];
      rz += rc[i] * zz[i];
    }
    write_pass_vec<T, MF>(camtab + (long long)CT * c, zz, pT + (long long)pass_vec_stride(MF) * c);
  }
  double v[1] = {rz};
  block_sum_all<1>(v);
  if (threadIdx.x == 0) dot_rz1[blockIdx.x] = v[0];
}

// Probe vectors: p = D^{-1/2} z^_k (z^ [C][K][9] FP32) into the solver's p
// and its pass form; zero for cameras without a scale.
// The coupling feature (off-diagonal norm summary of camera i's block row
// of S^ = D^{-1/2} S D^{-1/2}): kappa_i^2 = mean over COUPLING_PROBES
// Rademacher probes z of |(S^ z)_i - S^_ii z_i|^2, whose expectation is
// sum_{j != i} |S^_ij|_F^2.  Probe k's entry (c, a) is the sign bit of the
// SplitMix64 output for the counter k << 40 | c << 4 | a (Steele, Lea and
// Flood, OOPSLA 2014: golden-ratio increment, two xor-shift-multiply rounds,
// a final xor-shift), the oracle's generator.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double coupling_sign(int k, int c, int a) {
  const unsigned long long ctr = ((unsigned long long)k << 40) | ((unsigned long long)c << 4) | (unsigned long long)a;
  return (splitmix64(ctr) >> 63) ? -1.0 : 1.0;
}

// p = D^{-1/2} z_k (D = diag(S_ii) from the packed blocks), also in the
// passes' form.
template <typename T, bool MF>
static __global__ void k_coup_probe_in(int C, int k, const double* __restrict__ Sii, const T* __restrict__ camtab,
                                       double* __restrict__ p, T* __restrict__ pT) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double x[9];
  for (int a = 0; a < 9; ++a) {
    const double d = Sii[45LL * c + sym9(a, a)];
    x[a] = d > 0.0 ? coupling_sign(k, c, a) / sqrt(d) : 0.0;
    p[9LL * c + a] = x[a];
  }
  write_pass_vec<T, MF>(camtab + (long long)CT * c, x, pT + (long long)pass_vec_stride(MF) * c);
}

// kap[c] (+)= |D^{-1/2} q_c - S^_cc z_k,c|^2 with q = S p (k = 0 starts the sum).
static __global__ void k_coup_acc(int C, int k, const double* __restrict__ Sii, const double* __restrict__ q,
                                  double* __restrict__ kap) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const double* S = Sii + 45LL * c;
  double s[9], z[9];
  bool ok = true;
  for (int a = 0; a < 9; ++a) {
    const double d = S[sym9(a, a)];
    ok = ok && d > 0.0;
    s[a] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    z[a] = coupling_sign(k, c, a);
  }
  double acc = 0.0;
  if (ok) {
    for (int a = 0; a < 9; ++a) {
      double own = 0.0;
      for (int b = 0; b < 9; ++b) own += S[sym9_rt(a, b)] * s[a] * s[b] * z[b];
      const double off = q[9LL * c + a] * s[a] - own;
      acc += off * off;
    }
  }
  kap[c] = (k == 0 ? 0.0 : kap[c]) + acc;
}

template <typename T, bool MF>
static __global__ void k_probe_in(int C, int K, int k, const float* __restrict__ zhat, const double* __restrict__ D,
                           const T* __restrict__ camtab, double* __restrict__ p, T* __restrict__ pT) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double x[9];
  for (int a = 0; a < 9; ++a) {
    const double d = D[9LL * c + a];
    x[a] = d > 0.0 ? (double)zhat[(9LL * K) * c + 9 * k + a] / sqrt(d) : 0.0;
    p[9LL * c + a] = x[a];
  }
  write_pass_vec<T, MF>(camtab + (long long)CT * c, x, pT + (long long)pass_vec_stride(MF) * c);
}

// y^_k = D^{-1/2} (S p) into yhat [C][K][9].
static __global__ void k_probe_out(int C, int K, int k, const double* __restrict__ q, const double* __restrict__ D,
                            float* __restrict__ yhat) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  for (int a = 0; a < 9; ++a) {
    const double d = D[9LL * c + a];
    yhat[(9LL * K) * c + 9 * k + a] = d > 0.0 ? (float)(q[9LL * c + a] / sqrt(d)) : 0.f;
  }
}

// Slow-mode probe j: z^_j = D^{1/2} (x_ref - x) per camera component.
static __global__ void k_slow_diff(int C, int n, int j, const double* __restrict__ xref, const double* __restrict__ x,
                                   const double* __restrict__ D, float* __restrict__ zhat) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 9LL * C) return;
  const long long c = i / 9, a = i % 9;
  const double d = D[i];
  zhat[(9LL * n) * c + 9 * j + a] = d > 0.0 ? (float)((xref[i] - x[i]) * sqrt(d)) : 0.f;
}

// Scale each probe slot j to unit root-mean-square over the 9C components
// (one block; fixed-order sums).
static __global__ void k_slow_normalize(int C, int n, float* __restrict__ zhat) {
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (long long i = threadIdx.x; i < 9LL * C; i += blockDim.x) {
      const double v = zhat[(9LL * n) * (i / 9) + 9 * j + i % 9];
      s += v * v;
    }
    double v[1] = {s};
    block_sum_all<1>(v);
    const double rms = sqrt(v[0] / (9.0 * C));
    const float f = rms > 0.0 ? (float)(1.0 / rms) : 0.f;
    for (long long i = threadIdx.x; i < 9LL * C; i += blockDim.x) zhat[(9LL * n) * (i / 9) + 9 * j + i % 9] *= f;
    __syncthreads();
  }
}

}  // namespace ba
