// Learned proposal: a Fourier-space neural operator trained on descent trajectories.
//
// Network (per retained Fourier mode mp and sample s; F = NY*4 coefficients, W channels):
//   H0 = X[mp] E[mp]^T + bE;  Z_l = H_{l-1}[mp] (R_l[mp] + L_l)^T + b_l;
//   H_l = H_{l-1} + GELU(Z_l);  Y[mp] = H_L[mp] D[mp]^T + bD[mp].
// Activations are FP32 [MP][S][W]; every matrix product runs on the tensor cores in
// BF16 (operands rounded to bf16 when staged in shared memory) with FP32 accumulation
// (mma.sync m16n8k16).  The few reductions with a very long inner dimension (weight and
// bias gradients) sum FP32 partials in a fixed order.  Training uses Adam on FP32 master
// weights.  Proposals are judged by the residual norm of the descent (pcf_fno_propose).
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "pcf_ctx.h"

namespace pcf {

// ------------------------------------------------------------------ batched BF16 GEMM
// C[b](i,j) = alpha * sum_k A[b](i,k) B[b](k,j) + beta * C[b](i,j), all FP32 in memory with
// arbitrary strides (batch, row, col).
struct GemmArgs {
  const float* A;
  const float* B;
  float* C;
  long long sAb, sAi, sAk, sBb, sBk, sBj, sCb, sCi, sCj;
  int M, N, K;
  int nbatch, Klast;  // the last batch may have a shorter inner dimension (split-K chunks)
  float alpha, beta;
};

constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) k_gemm_bf16(GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 As[GBM][GBK + GPAD];
  __shared__ __align__(16) __nv_bfloat16 Bs[GBN][GBK + GPAD];
  const int bz = blockIdx.z;
  const float* A = g.A + bz * g.sAb;
  const float* B = g.B + bz * g.sBb;
  float* C = g.C + bz * g.sCb;
  const int i0 = blockIdx.y * GBM, j0 = blockIdx.x * GBN;
  const int Kb = (bz == g.nbatch - 1) ? g.Klast : g.K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gq = lane >> 2, tq = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  for (int k0 = 0; k0 < Kb; k0 += GBK) {
    for (int t = threadIdx.x; t < GBM * GBK; t += blockDim.x) {
      const int r = t / GBK, k = t - r * GBK;
      const int i = i0 + r, kk = k0 + k;
      const float v = (i < g.M && kk < Kb) ? A[i * g.sAi + kk * g.sAk] : 0.f;
      As[r][k] = __float2bfloat16_rn(v);
    }
    for (int t = threadIdx.x; t < GBN * GBK; t += blockDim.x) {
      const int cidx = t / GBK, k = t - cidx * GBK;
      const int j = j0 + cidx, kk = k0 + k;
      const float v = (j < g.N && kk < Kb) ? B[kk * g.sBk + j * g.sBj] : 0.f;
      Bs[cidx][k] = __float2bfloat16_rn(v);
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GBK; ks += 16) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int r = wm + a * 16 + gq;
        af[a][0] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * tq]);
        af[a][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * tq]);
        af[a][2] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * tq + 8]);
        af[a][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * tq + 8]);
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int cc = wn + b * 8 + gq;
        bf[b][0] = *reinterpret_cast<const uint32_t*>(&Bs[cc][ks + 2 * tq]);
        bf[b][1] = *reinterpret_cast<const uint32_t*>(&Bs[cc][ks + 2 * tq + 8]);
      }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) mma16816(acc[a][b], af[a], bf[b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int i = i0 + wm + a * 16 + gq + (h >= 2 ? 8 : 0);
        const int j = j0 + wn + b * 8 + 2 * tq + (h & 1);
        if (i < g.M && j < g.N) {
          float* cp = C + i * g.sCi + j * g.sCj;
          const float v = g.alpha * acc[a][b][h];
          *cp = g.beta == 0.f ? v : fmaf(g.beta, *cp, v);
        }
      }
}

void gemm(cudaStream_t s, GemmArgs g, int batch, int Klast = -1) {
  g.nbatch = batch;
  g.Klast = Klast < 0 ? g.K : Klast;
  dim3 grid((g.N + GBN - 1) / GBN, (g.M + GBM - 1) / GBM, batch);
  k_gemm_bf16<<<grid, 128, 0, s>>>(g);
}

// ------------------------------------------------------------------ elementwise and reductions
__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_df(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.3989422804014327f;
}

// Z += bias (per channel); Hn = H + GELU(Z)
__global__ void k_bias_resgelu(float* Z, const float* H, float* Hn, const float* bias, long long n, int C) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const float z = Z[t] + bias[t % C];
    Z[t] = z;
    Hn[t] = H[t] + gelu_f(z);
  }
}
// Y[mp][s][f] += bD[mp][f]
__global__ void k_add_mode_bias(float* Y, const float* bD, int MP, int S, int F) {
  const long long n = (long long)MP * S * F;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(t % F);
    const int mp = (int)(t / ((long long)S * F));
    Y[t] += bD[(size_t)mp * F + f];
  }
}
// dbD[mp][f] = sum_s dY[mp][s][f]
__global__ void k_mode_bias_grad(const float* dY, float* dbD, int MP, int S, int F) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < MP * F; t += gridDim.x * blockDim.x) {
    const int mp = t / F, f = t - mp * F;
    float a = 0.f;
    for (int s2 = 0; s2 < S; ++s2) a += dY[((size_t)mp * S + s2) * F + f];
    dbD[t] = a;
  }
}
__global__ void k_add_bias(float* Y, const float* bias, long long n, int C) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    Y[t] += bias[t % C];
}
// dZ = dH * GELU'(Z)
__global__ void k_gelu_back(const float* dH, const float* Z, float* dZ, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    dZ[t] = dH[t] * gelu_df(Z[t]);
}
// Wsum[mp] = R[mp] + L
__global__ void k_add_shared(const float* R, const float* Lm, float* out, long long n, int WW) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = R[t] + Lm[t % WW];
}
// dY = 2 (Y - T)/n, per-block partial sums of (Y - T)^2
__global__ void k_mse(const float* Y, const float* T, float* dY, long long n, double* part) {
  __shared__ double red[32];
  double s = 0.0;
  const float sc = 2.f / (float)n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const float d = Y[t] - T[t];
    dY[t] = sc * d;
    s += (double)d * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
    part[blockIdx.x] = a;
  }
}
// out[c] = sum over rows of X[rows][C] (column sums), partials per block then a final pass
__global__ void k_colsum_part(const float* X, long long rows, int C, float* part) {
  // block b sums rows b, b + G, ... for every column (C <= 64)
  __shared__ float red[256];
  for (int c0 = 0; c0 < C; c0 += 1) {
    float s = 0.f;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
         r += (long long)gridDim.x * blockDim.x)
      s += X[r * C + c0];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * C + c0] = red[0];
    __syncthreads();
  }
}
// out[e] = sum_g part[g][e] (+ out if accumulate)
__global__ void k_sum_parts(const float* part, int G, int E, float* out, int accumulate) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int gg = 0; gg < G; ++gg) s += part[(size_t)gg * E + e];
    out[e] = accumulate ? out[e] + s : s;
  }
}
// Adam on FP32 master weights
__global__ void k_adam(float* w, const float* gr, float* m, float* v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const float gg = gr[t];
    const float mm = b1 * m[t] + (1.f - b1) * gg;
    const float vv = b2 * v[t] + (1.f - b2) * gg * gg;
    m[t] = mm;
    v[t] = vv;
    w[t] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  }
}

// ------------------------------------------------------------------ state <-> features
// X[mp][b][n][4]: (Re v, Im v, Re eta, Im eta), eta = i kz u - i kx w; mean mode (u, w, 0, 0).
__global__ void k_features(LaunchInfo li, float* X, const float* sc, int B) {
  const int ny = li.insts[0].ny, nm = li.insts[0].nmodes;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)nm * B * ny;
       t += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(t % ny);
    const long long r = t / ny;
    const int b = (int)(r % B), mp = (int)(r / B);
    const Inst& I = li.insts[b];
    const int i = mp / I.Mz, p = mp - i * I.Mz;
    const double2* u = I.uhat;
    const double2 uu = u[((size_t)0 * nm + mp) * ny + n], vv = u[((size_t)1 * nm + mp) * ny + n],
                  ww = u[((size_t)2 * nm + mp) * ny + n];
    const float* s4 = sc + ((size_t)mp * ny + n) * 4;
    float4 o;
    if (mp == 0) {
      o = make_float4((float)(s4[0] * uu.x), (float)(s4[1] * ww.x), 0.f, 0.f);
    } else {
      const double a = I.kx[i], c = I.kz[p];
      o = make_float4((float)(s4[0] * vv.x), (float)(s4[1] * vv.y), (float)(s4[2] * (-c * uu.y + a * ww.y)),
                      (float)(s4[3] * (c * uu.x - a * ww.x)));
    }
    reinterpret_cast<float4*>(X)[t] = o;
  }
}

// psi of the proposal: raw features X/scale + Y/scale, independent modes only.
__global__ void k_features_to_psi(const float* X, const float* Y, const float* sc, const int* indep, int nindep,
                                  int ny, int Mz, int B, double* psi, long long psi_len) {
  const int N = ny - 1, segv = N - 3, sege = N - 1, seg = 2 * segv + 2 * sege;
  const long long total = (long long)B * (nindep + 1) * ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(t % ny);
    const long long r = t / ny;
    const int q = (int)(r % (nindep + 1)), b = (int)(r / (nindep + 1));
    const int mp = q < nindep ? indep[2 * q] * Mz + indep[2 * q + 1] : 0;
    const size_t xi = (((size_t)mp * B + b) * ny + n) * 4;
    double f[4];
    const float* s4 = sc + ((size_t)mp * ny + n) * 4;
    for (int k = 0; k < 4; ++k) f[k] = s4[k] > 0.f ? ((double)X[xi + k] + (double)Y[xi + k]) / (double)s4[k] : 0.0;
    double* o = psi + (size_t)b * psi_len;
    if (q < nindep) {
      o += (size_t)q * seg;
      if (n < segv) {
        o[n] = f[0];
        o[segv + n] = f[1];
      }
      if (n < sege) {
        o[2 * segv + n] = f[2];
        o[2 * segv + sege + n] = f[3];
      }
    } else if (n < sege) {
      o += (size_t)nindep * seg;
      o[n] = f[0];
      o[sege + n] = f[1];
    }
  }
}

// accepted instances take the proposal
__global__ void k_accept(double2* u, const double2* up, const double* J0, const double* J1, int* acc,
                         const long long* off, int B) {
  const int b = blockIdx.y;
  const bool take = isfinite(J1[b]) && J1[b] < J0[b];
  if (threadIdx.x == 0 && blockIdx.x == 0) acc[b] = take ? 1 : 0;
  if (!take) return;
  for (long long t = off[b] + blockIdx.x * (long long)blockDim.x + threadIdx.x; t < off[b + 1];
       t += (long long)gridDim.x * blockDim.x)
    u[t] = up[t];
}

}  // namespace pcf

using namespace pcf;

// ------------------------------------------------------------------ network object
struct pcf_fno {
  int MP, NY, W, L, CI;
  cudaStream_t s = nullptr;
  long long np = 0;
  std::vector<long long> off;  // parameter offsets: P bP Q bQ, then per layer R L K b
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  float* wsum = nullptr;
  int cap = 0;  // samples the activation buffers hold
  std::vector<float*> H, Z;
  float *Y = nullptr, *dY = nullptr, *dH = nullptr, *dZ = nullptr, *part = nullptr;
  double* dpart = nullptr;
  long long step = 0;
  // proposal buffers
  float *fX = nullptr, *fY = nullptr;
  double* fpsi = nullptr;
  double2* fu = nullptr;
  double *fJ0 = nullptr, *fJ1 = nullptr;
  int* facc = nullptr;
  long long* foff = nullptr;
  long long fcap = 0;
};

namespace {

enum { OE = 0, ObE = 1, OD = 2, ObD = 3 };
inline long long OR(const pcf_fno* f, int l) { return f->off[4 + 3 * l]; }
inline long long OL(const pcf_fno* f, int l) { return f->off[5 + 3 * l]; }
inline long long Ob(const pcf_fno* f, int l) { return f->off[6 + 3 * l]; }

constexpr int kPartBlocks = 256;

pcf_status ensure_cap(pcf_fno* f, int S) {
  if (S <= f->cap) return PCF_OK;
  for (float* p : f->H) cudaFree(p);
  for (float* p : f->Z) cudaFree(p);
  cudaFree(f->Y);
  cudaFree(f->dY);
  cudaFree(f->dH);
  cudaFree(f->dZ);
  f->H.assign(f->L + 1, nullptr);
  f->Z.assign(f->L, nullptr);
  const size_t act = (size_t)f->MP * S * f->W, io = (size_t)f->MP * S * f->NY * f->CI;
  for (auto& p : f->H)
    if (cudaMalloc(&p, act * sizeof(float))) return PCF_ENOMEM;
  for (auto& p : f->Z)
    if (cudaMalloc(&p, act * sizeof(float))) return PCF_ENOMEM;
  if (cudaMalloc(&f->Y, io * sizeof(float)) || cudaMalloc(&f->dY, io * sizeof(float)) ||
      cudaMalloc(&f->dH, act * sizeof(float)) || cudaMalloc(&f->dZ, act * sizeof(float)))
    return PCF_ENOMEM;
  f->cap = S;
  return PCF_OK;
}

GemmArgs ga(const float* A, long long sAb, long long sAi, long long sAk, const float* B, long long sBb, long long sBk,
            long long sBj, float* C, long long sCb, long long sCi, long long sCj, int M, int N, int K, float beta) {
  GemmArgs g;
  g.A = A; g.B = B; g.C = C;
  g.sAb = sAb; g.sAi = sAi; g.sAk = sAk; g.sBb = sBb; g.sBk = sBk; g.sBj = sBj;
  g.sCb = sCb; g.sCi = sCi; g.sCj = sCj;
  g.M = M; g.N = N; g.K = K; g.alpha = 1.f; g.beta = beta;
  return g;
}

int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 4096); }

// Y = network(X); keeps activations for the backward pass
void forward(pcf_fno* f, const float* X, int S, float* Y) {
  const int MP = f->MP, W = f->W, F = f->NY * f->CI;
  const long long act = (long long)MP * S * W;
  const float* w = f->w;
  // encoder per mode: H0[mp] = X[mp] E[mp]^T + bE
  gemm(f->s, ga(X, (long long)S * F, F, 1, w + f->off[OE], (long long)W * F, 1, F, f->H[0], (long long)S * W, W, 1,
                S, W, F, 0.f), MP);
  k_add_bias<<<grid_for(act), 256, 0, f->s>>>(f->H[0], w + f->off[ObE], act, W);
  for (int l = 0; l < f->L; ++l) {
    k_add_shared<<<grid_for((long long)MP * W * W), 256, 0, f->s>>>(w + OR(f, l), w + OL(f, l), f->wsum,
                                                                   (long long)MP * W * W, W * W);
    gemm(f->s, ga(f->H[l], (long long)S * W, W, 1, f->wsum, (long long)W * W, 1, W, f->Z[l], (long long)S * W, W, 1,
                  S, W, W, 0.f), MP);
    k_bias_resgelu<<<grid_for(act), 256, 0, f->s>>>(f->Z[l], f->H[l], f->H[l + 1], w + Ob(f, l), act, W);
  }
  // decoder per mode: Y[mp] = H_L[mp] D[mp]^T + bD[mp]
  gemm(f->s, ga(f->H[f->L], (long long)S * W, W, 1, w + f->off[OD], (long long)F * W, 1, W, Y, (long long)S * F, F, 1,
                S, F, W, 0.f), MP);
  k_add_mode_bias<<<grid_for((long long)MP * S * F), 256, 0, f->s>>>(Y, w + f->off[ObD], MP, S, F);
}

void colsum(pcf_fno* f, const float* X, long long rows, int C, float* out) {
  k_colsum_part<<<kPartBlocks, 256, 0, f->s>>>(X, rows, C, f->part);
  k_sum_parts<<<(C + 255) / 256, 256, 0, f->s>>>(f->part, kPartBlocks, C, out, 0);
}

// gradients of mean((Y - T)^2) into f->g; the loss via per-block partial sums
pcf_status backward(pcf_fno* f, const float* X, const float* T, int S, double* loss) {
  const int MP = f->MP, W = f->W, F = f->NY * f->CI;
  const long long act = (long long)MP * S * W, io = (long long)MP * S * F;
  float* g = f->g;
  const float* w = f->w;
  k_mse<<<kPartBlocks, 256, 0, f->s>>>(f->Y, T, f->dY, io, f->dpart);
  std::vector<double> hp(kPartBlocks);
  // decoder: dD[mp] = dY[mp]^T H_L[mp], dbD, dH = dY[mp] D[mp]
  gemm(f->s, ga(f->dY, (long long)S * F, 1, F, f->H[f->L], (long long)S * W, W, 1, g + f->off[OD], (long long)F * W,
                W, 1, F, W, S, 0.f), MP);
  k_mode_bias_grad<<<(MP * F + 255) / 256, 256, 0, f->s>>>(f->dY, g + f->off[ObD], MP, S, F);
  gemm(f->s, ga(f->dY, (long long)S * F, F, 1, w + f->off[OD], (long long)F * W, W, 1, f->dH, (long long)S * W, W, 1,
                S, W, F, 0.f), MP);
  for (int l = f->L - 1; l >= 0; --l) {
    k_gelu_back<<<grid_for(act), 256, 0, f->s>>>(f->dH, f->Z[l], f->dZ, act);
    colsum(f, f->dZ, (long long)MP * S, W, g + Ob(f, l));
    // dR[mp] = dZ[mp]^T H_{l-1}[mp]; dL = sum over modes
    gemm(f->s, ga(f->dZ, (long long)S * W, 1, W, f->H[l], (long long)S * W, W, 1, g + OR(f, l), (long long)W * W, W, 1,
                  W, W, S, 0.f), MP);
    k_sum_parts<<<(W * W + 255) / 256, 256, 0, f->s>>>(g + OR(f, l), MP, W * W, g + OL(f, l), 0);
    // residual: dH_{l-1} = dH_l + dZ[mp] Wsum[mp]
    k_add_shared<<<grid_for((long long)MP * W * W), 256, 0, f->s>>>(w + OR(f, l), w + OL(f, l), f->wsum,
                                                                   (long long)MP * W * W, W * W);
    gemm(f->s, ga(f->dZ, (long long)S * W, W, 1, f->wsum, (long long)W * W, W, 1, f->dH, (long long)S * W, W, 1, S, W,
                  W, 1.f), MP);
  }
  // encoder: dE[mp] = dH0[mp]^T X[mp], dbE
  gemm(f->s, ga(f->dH, (long long)S * W, 1, W, X, (long long)S * F, F, 1, g + f->off[OE], (long long)W * F, F, 1, W, F,
                S, 0.f), MP);
  colsum(f, f->dH, (long long)MP * S, W, g + f->off[ObE]);
  if (cudaMemcpyAsync(hp.data(), f->dpart, sizeof(double) * kPartBlocks, cudaMemcpyDeviceToHost, f->s) ||
      cudaStreamSynchronize(f->s))
    return PCF_ECUDA;
  double sum = 0.0;
  for (double x : hp) sum += x;
  *loss = sum / (double)io;
  return cudaGetLastError() == cudaSuccess ? PCF_OK : PCF_ECUDA;
}

}  // namespace

extern "C" {

pcf_status pcf_fno_create(int MP, int NY, int width, int layers, unsigned long long seed, void* stream, pcf_fno** out) {
  if (!out || MP < 1 || NY < 2 || width < 1 || width > 64 || layers < 1 || layers > 8) return PCF_EINVAL;
  pcf_fno* f = new pcf_fno();
  f->MP = MP; f->NY = NY; f->W = width; f->L = layers; f->CI = 4;
  f->s = (cudaStream_t)stream;
  const int W = width, F = NY * 4;
  long long o = 0;
  auto add = [&](long long n) { f->off.push_back(o); o += n; };
  add((long long)MP * W * F); add(W); add((long long)MP * F * W); add((long long)MP * F);
  for (int l = 0; l < layers; ++l) { add((long long)MP * W * W); add((long long)W * W); add(W); }
  f->np = o;
  // initial weights (Gaussian)
  std::vector<float> h(o, 0.f);
  std::mt19937_64 gen(seed);
  std::normal_distribution<double> nd;
  for (long long i = 0; i < (long long)MP * W * F; ++i) h[f->off[OE] + i] = (float)(nd(gen) / std::sqrt((double)F));
  for (long long i = 0; i < (long long)MP * F * W; ++i) h[f->off[OD] + i] = (float)(nd(gen) * 0.1 / std::sqrt((double)W));
  for (int l = 0; l < layers; ++l) {
    for (long long i = 0; i < (long long)MP * W * W; ++i) h[OR(f, l) + i] = (float)(nd(gen) * 0.5 / std::sqrt((double)W));
    for (long long i = 0; i < (long long)W * W; ++i) h[OL(f, l) + i] = (float)(nd(gen) * 0.5 / std::sqrt((double)W));
  }
  if (cudaMalloc(&f->w, o * sizeof(float)) || cudaMalloc(&f->g, o * sizeof(float)) ||
      cudaMalloc(&f->m, o * sizeof(float)) || cudaMalloc(&f->v, o * sizeof(float)) ||
      cudaMalloc(&f->wsum, (size_t)MP * W * W * sizeof(float)) ||
      cudaMalloc(&f->part, (size_t)kPartBlocks * 64 * 64 * sizeof(float)) ||
      cudaMalloc(&f->dpart, kPartBlocks * sizeof(double))) {
    pcf_fno_destroy(f);
    return PCF_ENOMEM;
  }
  if (cudaMemcpy(f->w, h.data(), o * sizeof(float), cudaMemcpyHostToDevice) ||
      cudaMemset(f->m, 0, o * sizeof(float)) || cudaMemset(f->v, 0, o * sizeof(float))) {
    pcf_fno_destroy(f);
    return PCF_ECUDA;
  }
  *out = f;
  return PCF_OK;
}

void pcf_fno_destroy(pcf_fno* f) {
  if (!f) return;
  if (f->s) cudaStreamSynchronize(f->s);
  for (float* p : f->H) cudaFree(p);
  for (float* p : f->Z) cudaFree(p);
  for (void* p : {(void*)f->w, (void*)f->g, (void*)f->m, (void*)f->v, (void*)f->wsum, (void*)f->Y, (void*)f->dY,
                  (void*)f->dH, (void*)f->dZ, (void*)f->part, (void*)f->dpart, (void*)f->fX, (void*)f->fY,
                  (void*)f->fpsi, (void*)f->fu, (void*)f->fJ0, (void*)f->fJ1, (void*)f->facc, (void*)f->foff})
    cudaFree(p);
  delete f;
}

long long pcf_fno_num_params(const pcf_fno* f) { return f ? f->np : 0; }

pcf_status pcf_fno_set_params(pcf_fno* f, const float* host) {
  if (!f || !host) return PCF_EINVAL;
  if (cudaMemcpy(f->w, host, f->np * sizeof(float), cudaMemcpyHostToDevice)) return PCF_ECUDA;
  return PCF_OK;
}

pcf_status pcf_fno_get_params(pcf_fno* f, float* host) {
  if (!f || !host) return PCF_EINVAL;
  if (cudaMemcpy(host, f->w, f->np * sizeof(float), cudaMemcpyDeviceToHost)) return PCF_ECUDA;
  return PCF_OK;
}

pcf_status pcf_fno_forward(pcf_fno* f, const float* X, int S, float* Y) {
  if (!f || !X || !Y || S < 1) return PCF_EINVAL;
  if (ensure_cap(f, S) != PCF_OK) return PCF_ENOMEM;
  forward(f, X, S, Y);
  return cudaGetLastError() == cudaSuccess ? PCF_OK : PCF_ECUDA;
}

pcf_status pcf_fno_loss_grad(pcf_fno* f, const float* X, const float* T, int S, double* loss, float* grad) {
  if (!f || !X || !T || S < 1) return PCF_EINVAL;
  if (ensure_cap(f, S) != PCF_OK) return PCF_ENOMEM;
  forward(f, X, S, f->Y);
  double l = 0.0;
  const pcf_status st = backward(f, X, T, S, &l);
  if (st != PCF_OK) return st;
  if (loss) *loss = l;
  if (grad && cudaMemcpy(grad, f->g, f->np * sizeof(float), cudaMemcpyDeviceToDevice)) return PCF_ECUDA;
  return PCF_OK;
}

pcf_status pcf_fno_train_step(pcf_fno* f, const float* X, const float* T, int S, float lr, double* loss) {
  if (!f || !X || !T || S < 1 || !(lr > 0)) return PCF_EINVAL;
  if (ensure_cap(f, S) != PCF_OK) return PCF_ENOMEM;
  forward(f, X, S, f->Y);
  double l = 0.0;
  const pcf_status st = backward(f, X, T, S, &l);
  if (st != PCF_OK) return st;
  f->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)f->step), c2 = 1.f - std::pow(b2, (float)f->step);
  k_adam<<<grid_for(f->np), 256, 0, f->s>>>(f->w, f->g, f->m, f->v, f->np, lr, b1, b2, 1e-8f, c1, c2);
  if (loss) *loss = l;
  return cudaGetLastError() == cudaSuccess ? PCF_OK : PCF_ECUDA;
}

pcf_status pcf_fno_features(pcf_ctx* c, const double* u_hat, float* X, const float* scale) {
  if (!c || !u_hat || !X || !c->uniform) return PCF_EINVAL;
  for (int b = 0; b < c->B; ++b) c->hinst[b].uhat = (double2*)u_hat + c->state_off[b];
  if (cudaMemcpyAsync(c->dinst, c->hinst.data(), sizeof(Inst) * c->B, cudaMemcpyHostToDevice, c->user))
    return PCF_ECUDA;
  const long long n = (long long)c->nm * c->B * c->prm.ny;
  if (!scale) return PCF_EINVAL;
  k_features<<<grid_for(n), 256, 0, c->user>>>(LaunchInfo{c->dinst, c->pre_inst, c->B}, X, scale, c->B);
  return cudaGetLastError() == cudaSuccess ? PCF_OK : PCF_ECUDA;
}

// Proposal step of the learned acceleration: u' = completion(features(u) + network(features(u))).
// With relax_steps = k > 0 both u and u' then take k plain descent steps (dtau) and are
// compared there; instance b keeps the proposal's branch iff its residual norm is lower.
pcf_status pcf_fno_propose(pcf_ctx* c, pcf_fno* f, double* u_hat, const float* scale, int relax_steps, double dtau,
                           int* accepted, double* J_before, double* J_after) {
  if (!c || !f || !u_hat || !c->uniform || !scale || relax_steps < 0 || !(dtau > 0)) return PCF_EINVAL;
  if (f->MP != c->nm || f->NY != c->prm.ny) return PCF_EINVAL;
  const int B = c->B;
  const long long nx = (long long)c->nm * B * c->prm.ny * 4;
  if (f->fcap < B) {
    for (void* p : {(void*)f->fX, (void*)f->fY, (void*)f->fpsi, (void*)f->fu, (void*)f->fJ0, (void*)f->fJ1,
                    (void*)f->facc, (void*)f->foff})
      cudaFree(p);
    const long long plen = pcf_psi_len(c->prm.nx, c->prm.ny, c->prm.nz);
    if (cudaMalloc(&f->fX, nx * sizeof(float)) || cudaMalloc(&f->fY, nx * sizeof(float)) ||
        cudaMalloc(&f->fpsi, (size_t)B * plen * sizeof(double)) ||
        cudaMalloc(&f->fu, (size_t)c->total_state * sizeof(double2)) || cudaMalloc(&f->fJ0, B * sizeof(double)) ||
        cudaMalloc(&f->fJ1, B * sizeof(double)) || cudaMalloc(&f->facc, B * sizeof(int)) ||
        cudaMalloc(&f->foff, (B + 1) * sizeof(long long)))
      return PCF_ENOMEM;
    if (cudaMemcpy(f->foff, c->state_off.data(), (B + 1) * sizeof(long long), cudaMemcpyHostToDevice))
      return PCF_ECUDA;
    f->fcap = B;
  }
  pcf_status st = pcf_fno_features(c, u_hat, f->fX, scale);
  if (st != PCF_OK) return st;
  cudaStream_t keep = f->s;
  f->s = c->user;
  st = pcf_fno_forward(f, f->fX, B, f->fY);
  f->s = keep;
  if (st != PCF_OK) return st;
  // completion of the proposal through the snapshot coordinates (pcf_snapshot builds the
  // independent-mode table on first use; its output is overwritten below)
  {
    st = pcf_snapshot(c, u_hat, f->fpsi);
    if (st != PCF_OK) return st;
    const int nind = c->nindep;
    const long long plen = c->psi_len;
    const long long tot = (long long)B * (nind + 1) * c->prm.ny;
    k_features_to_psi<<<grid_for(tot), 256, 0, c->user>>>(f->fX, f->fY, scale, c->d_indep, nind, c->prm.ny,
                                                          c->Mz, B, f->fpsi, plen);
    if ((st = pcf_from_snapshot(c, f->fpsi, (double*)f->fu)) != PCF_OK) return st;
  }
  if (relax_steps > 0) {
    if ((st = pcf_descent_step(c, (double*)f->fu, dtau, relax_steps, nullptr)) != PCF_OK) return st;
    if ((st = pcf_descent_step(c, u_hat, dtau, relax_steps, nullptr)) != PCF_OK) return st;
  }
  if ((st = pcf_residual(c, u_hat, (double*)c->r_int, f->fJ0)) != PCF_OK) return st;
  if ((st = pcf_residual(c, (const double*)f->fu, (double*)c->r_int, f->fJ1)) != PCF_OK) return st;
  k_accept<<<dim3(64, B), 256, 0, c->user>>>((double2*)u_hat, f->fu, f->fJ0, f->fJ1, f->facc, f->foff, B);
  if (cudaGetLastError()) return PCF_ECUDA;
  if (accepted && cudaMemcpyAsync(accepted, f->facc, B * sizeof(int), cudaMemcpyDeviceToHost, c->user)) return PCF_ECUDA;
  if (J_before && cudaMemcpyAsync(J_before, f->fJ0, B * sizeof(double), cudaMemcpyDeviceToHost, c->user))
    return PCF_ECUDA;
  if (J_after && cudaMemcpyAsync(J_after, f->fJ1, B * sizeof(double), cudaMemcpyDeviceToHost, c->user))
    return PCF_ECUDA;
  if (cudaStreamSynchronize(c->user)) return PCF_ECUDA;
  return PCF_OK;
}

}  // extern "C"
