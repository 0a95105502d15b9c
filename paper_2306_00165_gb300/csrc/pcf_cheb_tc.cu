// Chebyshev transforms of the mixed-precision form on the tensor cores.
//
// In y every field column (one Fourier mode, real or imaginary part) is multiplied by a
// dense ny x ny matrix: values from coefficients (T_n(y_j)), y-derivative values from
// coefficients (T'_n(y_j)), coefficients from values (the DCT-I inverse).  Across all modes
// and components these are GEMMs  Out[M x ncol] = A[M x K] B[K x ncol]  with M = K = ny.
// They run as split-BF16 products on the tensor cores with FP32 accumulation: each operand
// x is split into x_hi = bf16(x) and x_lo = bf16(x - x_hi), and
//   A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi,
// which keeps about 16 significant bits of each product.  The contraction is memory bound
// (about 2 ny flops per 8 bytes moved), so mma.sync tiles of 16 x 8 x 16 suffice; one CTA
// holds the whole (padded) matrix and a 64-column tile of B in shared memory.
#include <cuda_bf16.h>

#include "pcf_ctx.h"

namespace pcf {

constexpr int kTcCols = 64;     // columns of B per CTA
constexpr int kTcThreads = 256;

__host__ __device__ inline int pad16(int n) { return (n + 15) & ~15; }

size_t smem_cheb_tc(int ny) {
  const int P = pad16(ny);
  return (size_t)2 * P * P * 2 + (size_t)2 * kTcCols * P * 2;
}

__device__ __forceinline__ void mma_bf16(float* c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16* hi, __nv_bfloat16* lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  *hi = h;
  *lo = __float2bfloat16_rn(x - __bfloat162float(h));
}

// Shared core: A (hi, lo) [P][P] and B (hi, lo) [kTcCols][P] (k contiguous) are in shared
// memory; computes the P x kTcCols tile and hands each output (row, col) to store().
template <class Store>
__device__ __forceinline__ void tc_tile(const __nv_bfloat16* Ah, const __nv_bfloat16* Al, const __nv_bfloat16* Bh,
                                        const __nv_bfloat16* Bl, int P, int Mrows, Store store) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int mt = P / 16, nt = kTcCols / 8;
  for (int tile = warp; tile < mt * nt; tile += kTcThreads / 32) {
    const int r0 = (tile / nt) * 16, c0 = (tile % nt) * 8;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < P; k0 += 16) {
      const int ka = k0 + 2 * t;
      const uint32_t* rowa0h = reinterpret_cast<const uint32_t*>(Ah + (size_t)(r0 + g) * P + ka);
      const uint32_t* rowa1h = reinterpret_cast<const uint32_t*>(Ah + (size_t)(r0 + g + 8) * P + ka);
      const uint32_t* rowa0l = reinterpret_cast<const uint32_t*>(Al + (size_t)(r0 + g) * P + ka);
      const uint32_t* rowa1l = reinterpret_cast<const uint32_t*>(Al + (size_t)(r0 + g + 8) * P + ka);
      const uint32_t* colbh = reinterpret_cast<const uint32_t*>(Bh + (size_t)(c0 + g) * P + ka);
      const uint32_t* colbl = reinterpret_cast<const uint32_t*>(Bl + (size_t)(c0 + g) * P + ka);
      const uint32_t ah0 = rowa0h[0], ah1 = rowa1h[0], ah2 = rowa0h[4], ah3 = rowa1h[4];
      const uint32_t al0 = rowa0l[0], al1 = rowa1l[0], al2 = rowa0l[4], al3 = rowa1l[4];
      const uint32_t bh0 = colbh[0], bh1 = colbh[4], bl0 = colbl[0], bl1 = colbl[4];
      mma_bf16(acc, ah0, ah1, ah2, ah3, bh0, bh1);
      mma_bf16(acc, ah0, ah1, ah2, ah3, bl0, bl1);
      mma_bf16(acc, al0, al1, al2, al3, bh0, bh1);
    }
    const int row0 = r0 + g, row1 = r0 + g + 8, col = c0 + 2 * t;
    if (row0 < Mrows) {
      store(row0, col, acc[0]);
      store(row0, col + 1, acc[1]);
    }
    if (row1 < Mrows) {
      store(row1, col, acc[2]);
      store(row1, col + 1, acc[3]);
    }
  }
}

__device__ __forceinline__ void load_matrix(const __nv_bfloat16* src_hi, const __nv_bfloat16* src_lo,
                                            __nv_bfloat16* Ah, __nv_bfloat16* Al, int P) {
  const uint4* sh = reinterpret_cast<const uint4*>(src_hi);
  const uint4* sl = reinterpret_cast<const uint4*>(src_lo);
  uint4* dh = reinterpret_cast<uint4*>(Ah);
  uint4* dl = reinterpret_cast<uint4*>(Al);
  const int n16 = P * P * 2 / 16;
  for (int i = threadIdx.x; i < n16; i += blockDim.x) {
    dh[i] = sh[i];
    dl[i] = sl[i];
  }
}

// Synthesis: yvf[slot][q][j][col] = sum_n M_q[j][n] a_c(q)[n][col], q = V_u V_v V_w W_u W_w,
// a from the FP64 state (uhat for slot 0, rhat for slot 1).  CTA = (instance, q, column tile).
__global__ void __launch_bounds__(kTcThreads) k_cheb_synth_tc(LaunchInfo li, int slot) {
  extern __shared__ __align__(16) unsigned char smraw[];
  int local;
  const int b = find_inst(li, blockIdx.x, &local);
  const Inst& I = li.insts[b];
  if (I.active && !*I.active) return;
  const int ny = I.ny, nm = I.nmodes, P = pad16(ny), ncol = 2 * nm;
  const int ntiles = (ncol + kTcCols - 1) / kTcCols;
  const int q = local / ntiles, tile = local - q * ntiles;
  const int c = q < 3 ? q : (q == 3 ? 0 : 2);
  __nv_bfloat16* Ah = reinterpret_cast<__nv_bfloat16*>(smraw);
  __nv_bfloat16* Al = Ah + P * P;
  __nv_bfloat16* Bh = Al + P * P;
  __nv_bfloat16* Bl = Bh + kTcCols * P;
  const int mat = q < 3 ? 0 : 1;
  const __nv_bfloat16* A = reinterpret_cast<const __nv_bfloat16*>(I.tcA);
  load_matrix(A + (size_t)(2 * mat) * P * P, A + (size_t)(2 * mat + 1) * P * P, Ah, Al, P);
  const double2* a = (slot == 0 ? I.uhat : I.rhat) + (size_t)c * nm * ny;
  const int col0 = tile * kTcCols;
  for (int i = threadIdx.x; i < kTcCols * P; i += blockDim.x) {
    const int cc = i / P, n = i - cc * P, col = col0 + cc;
    float x = 0.f;
    if (n < ny && col < ncol) {
      const double2 v = a[(size_t)(col >> 1) * ny + n];
      x = (float)((col & 1) ? v.y : v.x);
    }
    split_bf16(x, Bh + i, Bl + i);
  }
  __syncthreads();
  float* out = reinterpret_cast<float*>(I.yvf + (((size_t)slot * kFieldsY + q) * ny) * nm);
  tc_tile(Ah, Al, Bh, Bl, P, ny, [&](int j, int cc, float v) {
    const int col = col0 + cc;
    if (col < ncol) out[(size_t)j * ncol + col] = v;
  });
}

// Analysis: xzc[c][n][col] = sum_j Cinv[n][j] xzf[c][j][col].  CTA = (instance, c, column tile).
__global__ void __launch_bounds__(kTcThreads) k_cheb_analysis_tc(LaunchInfo li) {
  extern __shared__ __align__(16) unsigned char smraw[];
  int local;
  const int b = find_inst(li, blockIdx.x, &local);
  const Inst& I = li.insts[b];
  if (I.active && !*I.active) return;
  const int ny = I.ny, nm = I.nmodes, P = pad16(ny), ncol = 2 * nm;
  const int ntiles = (ncol + kTcCols - 1) / kTcCols;
  const int c = local / ntiles, tile = local - c * ntiles;
  __nv_bfloat16* Ah = reinterpret_cast<__nv_bfloat16*>(smraw);
  __nv_bfloat16* Al = Ah + P * P;
  __nv_bfloat16* Bh = Al + P * P;
  __nv_bfloat16* Bl = Bh + kTcCols * P;
  const __nv_bfloat16* A = reinterpret_cast<const __nv_bfloat16*>(I.tcA);
  load_matrix(A + (size_t)4 * P * P, A + (size_t)5 * P * P, Ah, Al, P);
  const float* src = reinterpret_cast<const float*>(I.xzf + (size_t)c * ny * nm);
  const int col0 = tile * kTcCols;
  for (int i = threadIdx.x; i < kTcCols * P; i += blockDim.x) {
    const int j = i / kTcCols, cc = i - j * kTcCols, col = col0 + cc;  // coalesced along col
    float x = 0.f;
    if (j < ny && col < ncol) x = src[(size_t)j * ncol + col];
    split_bf16(x, Bh + (size_t)cc * P + j, Bl + (size_t)cc * P + j);
  }
  __syncthreads();
  float* out = reinterpret_cast<float*>(I.xzc + (size_t)c * ny * nm);
  tc_tile(Ah, Al, Bh, Bl, P, ny, [&](int n, int cc, float v) {
    const int col = col0 + cc;
    if (col < ncol) out[(size_t)n * ncol + col] = v;
  });
}

void launch_cheb_synth_tc(int ctas, size_t smem, cudaStream_t s, LaunchInfo li, int slot) {
  k_cheb_synth_tc<<<ctas, kTcThreads, smem, s>>>(li, slot);
}
void launch_cheb_analysis_tc(int ctas, size_t smem, cudaStream_t s, LaunchInfo li) {
  k_cheb_analysis_tc<<<ctas, kTcThreads, smem, s>>>(li);
}
cudaError_t set_cheb_tc_smem(size_t smem) {
  cudaError_t e = raise_smem_limit((const void*)k_cheb_synth_tc, smem);
  if (e) return e;
  return raise_smem_limit((const void*)k_cheb_analysis_tc, smem);
}
int cheb_tc_tiles(int nmodes) { return (2 * nmodes + kTcCols - 1) / kTcCols; }

}  // namespace pcf
