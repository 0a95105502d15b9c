// Chebyshev transforms of the mixed-precision form on the 5th-generation tensor cores
// (tcgen05): the split-BF16 contraction Out = A B with the accumulator in tensor memory.
//
// Per CTA one tile D[128 x 64] = A[128 x P] B[P x 64] of a y-transform (P = ny rounded up to
// 16; A rows >= P and B rows >= ny are zero):
//   analysis   xzc[c][n][col] = sum_j Cinv[n][j] xzf[c][j][col]    (A = Cinv, B from FP32)
//   synthesis  yvf[q][j][col] = sum_n M_q[j][n] a_c(q)[n][col]      (A = C or C', B from the
//              FP64 state, col = 2 mode + re/im)
// Each operand x is split into x_hi = bf16(x) and x_lo = bf16(x - x_hi), and
// A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi: three MMAs of kind::f16 (BF16 inputs, FP32
// accumulation) per 16-wide K step, issued by one thread into one TMEM accumulator.
//
// Operands live in shared memory in the no-swizzle K-major layout of core matrices (8 rows of
// 16 bytes each, 128 contiguous bytes): the core matrix of rows 8g..8g+7 and K elements
// 8kc..8kc+7 of an R-row operand starts at byte (kc R/8 + g) 128, so the descriptor's
// leading-dimension byte offset (next core matrix along K) is R/8 * 128 and its
// stride-dimension byte offset (next 8 rows) is 128.  Every 16-byte chunk of a row (8
// consecutive K elements) is one shared-memory store.
//
// The accumulator (128 lanes x 64 FP32 columns) is read back by the eight warps (warp w owns
// TMEM lanes 32 (w mod 4) .. + 31, i.e. output rows, and columns 32 (w / 4) .. + 31), staged
// in shared memory and written out row by row with coalesced stores.  The wait for the MMAs is bounded: after about two seconds the
// CTA gives up, writes NaN to its outputs (the residual norm then reports PCF_ENAN), frees its
// tensor memory and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "pcf_ctx.h"

namespace pcf {

namespace {

constexpr int kT5Rows = 128;    // MMA M (output rows, padded)
constexpr int kT5Cols = 64;     // MMA N (columns per CTA)
constexpr int kT5Threads = 256;  // 8 warps: warp w reads TMEM lanes 32 (w % 4).., column half w / 4

__host__ __device__ inline int pad16_5(int n) { return (n + 15) & ~15; }

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of tcgen05 (no swizzle): start address, leading- and
// stride-dimension byte offsets (each encoded >> 4), and the fixed 0b001 at bits 46-48.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | ((uint64_t)1 << 46);
}

// Byte offset of the 16-byte chunk (row r, K elements 8kc..8kc+7) of an R-row operand.
__device__ __forceinline__ uint32_t chunk_off(int r, int kc, int R) {
  return (uint32_t)(kc * (R >> 3) + (r >> 3)) * 128u + (uint32_t)(r & 7) * 16u;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
  return (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
}

// Split 8 FP32 values into their BF16 high parts and the BF16 of the remainders, packed.
__device__ __forceinline__ void split8(const float* v, uint4& hi, uint4& lo) {
  float h[8], l[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const __nv_bfloat16 b = __float2bfloat16_rn(v[i]);
    h[i] = __bfloat162float(b);
    l[i] = v[i] - h[i];
  }
  hi = make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]), pack_bf16(h[6], h[7]));
  lo = make_uint4(pack_bf16(l[0], l[1]), pack_bf16(l[2], l[3]), pack_bf16(l[4], l[5]), pack_bf16(l[6], l[7]));
}

}  // namespace

// A region (A hi and lo, later the D staging), then B hi and lo, then the mbarrier and the
// TMEM address slot.
__host__ __device__ inline size_t t5_aregion(int P) {
  const size_t a = (size_t)2 * kT5Rows * P * 2;
  const size_t stage = (size_t)kT5Rows * (kT5Cols + 1) * 4;
  return a > stage ? a : stage;
}

size_t smem_cheb_tc05(int ny) {
  const int P = pad16_5(ny);
  return t5_aregion(P) + (size_t)2 * kT5Cols * P * 2 + 64;
}

// CTA = (instance, output field q or component c, tile of 64 columns); same CTA map as the
// mma.sync kernels.  SYN: synthesis of slot `slot`, else analysis.
template <bool SYN>
__global__ void __launch_bounds__(kT5Threads) k_cheb_tc05(LaunchInfo li, int slot) {
  extern __shared__ __align__(128) unsigned char sm5[];
  __shared__ int ok;
  int local;
  const int b = find_inst(li, blockIdx.x, &local);
  const Inst& I = li.insts[b];
  if (I.active && !*I.active) return;
  const int ny = I.ny, nm = I.nmodes, P = pad16_5(ny), KC = P >> 3, ncol = 2 * nm;
  const int ntiles = (ncol + kT5Cols - 1) / kT5Cols;
  const int q = local / ntiles, tile = local - q * ntiles;
  const int col0 = tile * kT5Cols;
  const size_t abytes = (size_t)kT5Rows * P * 2, bbytes = (size_t)kT5Cols * P * 2;
  unsigned char* sAh = sm5;
  unsigned char* sAl = sm5 + abytes;
  unsigned char* sBh = sm5 + t5_aregion(P);
  unsigned char* sBl = sBh + bbytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sBl + bbytes);  // MMA completion
  uint64_t* abar = mbar + 1;                                      // A operand arrival
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  float* sD = reinterpret_cast<float*>(sm5);
  // A: analysis Cinv (matrix 2), synthesis C (0) for the values, C' (1) for the y-derivatives.
  // Its hi and lo parts are stored in global memory as images of the shared-memory region
  // (core-matrix layout), and one thread moves them with two bulk copies on the TMA engine
  // while the CTA splits its B tile.
  const int mat = SYN ? (q < 3 ? 0 : 1) : 2;
  if (threadIdx.x == 0) {
    ok = 1;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(abar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const unsigned char* img = static_cast<const unsigned char*>(I.tcA5) + (size_t)(2 * mat) * abytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(abar)),
                 "r"((uint32_t)(2 * abytes))
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(sAh)),
        "l"(img), "r"((uint32_t)abytes), "r"(smem_addr(abar))
        : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(sAl)),
        "l"(img + abytes), "r"((uint32_t)abytes), "r"(smem_addr(abar))
        : "memory");
  }
  // B: 8 consecutive K elements of one column per task, split into BF16 high and low parts
  for (int t = threadIdx.x; t < kT5Cols * KC; t += blockDim.x) {
    const int kc = t / kT5Cols, cc = t - kc * kT5Cols, col = col0 + cc;
    float v[8];
    if (SYN) {
      const int c = q < 3 ? q : (q == 3 ? 0 : 2);
      const double2* a = (slot == 0 ? I.uhat : I.rhat) + (size_t)c * nm * ny + (size_t)(col >> 1) * ny;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int n = 8 * kc + i;
        float x = 0.f;
        if (col < ncol && n < ny) {
          const double2 z = a[n];
          x = (float)((col & 1) ? z.y : z.x);
        }
        v[i] = x;
      }
    } else {
      const float* src = reinterpret_cast<const float*>(I.xzf + (size_t)q * ny * nm);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int j = 8 * kc + i;
        v[i] = (col < ncol && j < ny) ? src[(size_t)j * ncol + col] : 0.f;
      }
    }
    uint4 h, l;
    split8(v, h, l);
    const uint32_t o = chunk_off(cc, kc, kT5Cols);
    *reinterpret_cast<uint4*>(sBh + o) = h;
    *reinterpret_cast<uint4*>(sBl + o) = l;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_addr(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  // the A operand must have arrived before the MMAs read it (bounded wait, as below)
  bool a_ok = true;
  if (threadIdx.x == 0) {
    uint32_t arrived = 0;
    const long long ta = clock64();
    while (!arrived) {
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(arrived)
          : "r"(smem_addr(abar)), "r"(0u)
          : "memory");
      if (!arrived && clock64() - ta > 4000000000LL) break;
    }
    if (!arrived) {
      // no MMAs: release the waiters below through the completion barrier, outputs NaN
      a_ok = false;
      ok = 0;
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(mbar)) : "memory");
    }
  }
  if (threadIdx.x == 0 && a_ok) {
    // kind::f16 instruction descriptor: FP32 accumulator (bits 4-5 = 1), BF16 A and B (bits
    // 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kT5Cols >> 3) << 17) |
                           ((uint32_t)(kT5Rows >> 4) << 24);
    const uint32_t albo = (kT5Rows / 8) * 128, blbo = (kT5Cols / 8) * 128, sbo = 128;
    for (int s = 0; s < P / 16; ++s) {
      const uint32_t ao = (uint32_t)(2 * s) * albo, bo = (uint32_t)(2 * s) * blbo;
      const uint64_t ah = umma_desc(smem_addr(sAh) + ao, albo, sbo), al = umma_desc(smem_addr(sAl) + ao, albo, sbo);
      const uint64_t bh = umma_desc(smem_addr(sBh) + bo, blbo, sbo), bl = umma_desc(smem_addr(sBl) + bo, blbo, sbo);
      const uint64_t da[3] = {ah, ah, al}, db[3] = {bh, bl, bh};
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const uint32_t acc = (s > 0 || p > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred q;\nsetp.ne.b32 q, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem),
            "l"(da[p]), "l"(db[p]), "r"(idesc), "r"(acc));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
                 : "memory");
  }
  // bounded wait for the MMAs (about two seconds at the boost clock)
  uint32_t done = 0;
  const long long t0 = clock64();
  while (!done) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(0u)
        : "memory");
    if (!done && clock64() - t0 > 4000000000LL) {
      ok = 0;
      break;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // tcgen05.ld is warp-collective: read the accumulator only if every lane saw the MMAs finish
  if (__all_sync(0xffffffffu, done && ok)) {
    {
      const int quarter = warp & 3, half = warp >> 2;
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + 32u * half;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float* row = sD + (size_t)(32 * quarter + lane) * (kT5Cols + 1) + 32 * half;
#pragma unroll
      for (int c = 0; c < 32; ++c) row[c] = __uint_as_float(r[c]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
  float* out = SYN ? reinterpret_cast<float*>(I.yvf + (((size_t)slot * kFieldsY + q) * ny) * nm)
                   : reinterpret_cast<float*>(I.xzc + (size_t)q * ny * nm);
  const int good = ok;
  for (int t = threadIdx.x; t < ny * kT5Cols; t += blockDim.x) {
    const int m = t / kT5Cols, cc = t - m * kT5Cols, col = col0 + cc;
    if (col < ncol) out[(size_t)m * ncol + col] = good ? sD[(size_t)m * (kT5Cols + 1) + cc] : __int_as_float(0x7fc00000);
  }
}

void launch_cheb_synth_tc05(int ctas, size_t smem, cudaStream_t s, LaunchInfo li, int slot) {
  k_cheb_tc05<true><<<ctas, kT5Threads, smem, s>>>(li, slot);
}
void launch_cheb_analysis_tc05(int ctas, size_t smem, cudaStream_t s, LaunchInfo li) {
  k_cheb_tc05<false><<<ctas, kT5Threads, smem, s>>>(li, 0);
}
cudaError_t set_cheb_tc05_smem(size_t smem) {
  cudaError_t e = raise_smem_limit((const void*)k_cheb_tc05<true>, smem);
  if (e) return e;
  return raise_smem_limit((const void*)k_cheb_tc05<false>, smem);
}

}  // namespace pcf
