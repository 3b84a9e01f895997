// Inner F-apply of the mixed-precision PCGP for subdomains that share their
// shape's elastic factor: with S = (K^+)_{boundary,boundary} of the shape (formed
// once in FP64, stored FP32), the subdomain part of F = B K^+ B^T for all such
// subdomains is one GEMM  Y = X S,  X[k] = B^T lam gathered onto the box
// boundary dofs of subdomain k (zero off its interface).  S is symmetric.
//
// The GEMM runs on the tensor cores (tcgen05.mma, kind::tf32, accumulator in
// tensor memory) with each FP32 operand split into two TF32 parts,
// a = a_hi + a_lo, and D += A_hi B_hi + A_hi B_lo + A_lo B_hi, which keeps the
// product at FP32 accuracy (the dropped A_lo B_lo term is ~2^-22 relative).
//
// Operand tiles are stored in global memory already in the shared-memory layout
// the MMA reads (no swizzle, K-major "core matrices" of 8 rows x 16 bytes), so
// one pipeline stage is four contiguous 1-D bulk copies:
//   A (X) tile: 128 rows (subdomains) x 32 columns (dofs), core matrix (kg, mg)
//               at byte (kg * 16 + mg) * 128;  B (S) tile: kTN = 32 rows x 32 columns,
//               core matrix (kg, ng) at byte (kg * 4 + ng) * 128;
// row r of a core matrix holds 4 consecutive K elements (16 bytes).
#include "async_common.cuh"
#include "dev.h"
#include "dual_common.cuh"

namespace tfeti {

namespace {

constexpr int kTM = 128, kTN = 32, kTK = 32, kStages = 4;
constexpr uint32_t kABytes = kTM * kTK * 4, kBBytes = kTN * kTK * 4;
constexpr uint32_t kStageBytes = 2 * kABytes + 2 * kBBytes;
constexpr uint32_t kTmemCols = kTN;  // FP32 accumulator columns (a power of two >= 32)

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = tf32_round(x);
  lo = tf32_round(x - hi);
}

// Offset (floats) of element (row, col) inside an A tile (rows < 128) or a B tile
// (rows < 64, groups = 8), col < 32.
__device__ __forceinline__ int tile_off(int row, int col, int groups) {
  return (((col >> 2) * groups + (row >> 3)) * 8 + (row & 7)) * 4 + (col & 3);
}

// X tiles: Xhi/Xlo[(mt * nk + ks) * 4096 + tile_off(r, c, 16)] for subdomain
// sub_list[mt * 128 + r] and boundary dof ks * 32 + c (zero beyond n_list, n_bd).
__global__ void k_schur_gather_tc(DevMesh M, const int* __restrict__ sub_list, int n_list, int n_bd, int nk,
                                  const double* __restrict__ lam, float* Xhi, float* Xlo) {
  const long long ncol = (long long)nk * kTK;
  const int n_mt = (n_list + kTM - 1) / kTM;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)n_mt * kTM * ncol) return;
  const int k = (int)(idx / ncol), j = (int)(idx % ncol);
  float v = 0.0f;
  if (k < n_list && j < n_bd) {
    const SubDev& S = M.subs[sub_list[k]];
    const int sl = M.sub_b2s[S.b2s_off + j / 3];
    if (sl >= 0) v = (float)bt_at_slot(M, lam, (long long)sl + j % 3);
  }
  const int mt = k / kTM, ks = j / kTK;
  const long long o = ((long long)mt * nk + ks) * (kTM * kTK) + tile_off(k % kTM, j % kTK, kTM / 8);
  float hi, lo;
  split_tf32(v, hi, lo);
  Xhi[o] = hi;
  Xlo[o] = lo;
}

// S tiles from the FP32 block S32 (S32[j * n_bd + i] = S[i][j]).
__global__ void k_schur_tile_S(const float* __restrict__ S32, int n_bd, int nk, float* Shi, float* Slo) {
  const long long ncol = (long long)nk * kTK;
  const int n_nt = (n_bd + kTN - 1) / kTN;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)n_nt * kTN * ncol) return;
  const int i = (int)(idx / ncol), j = (int)(idx % ncol);
  const float v = (i < n_bd && j < n_bd) ? S32[(long long)j * n_bd + i] : 0.0f;
  const int nt = i / kTN, ks = j / kTK;
  const long long o = ((long long)nt * nk + ks) * (kTN * kTK) + tile_off(i % kTN, j % kTK, kTN / 8);
  float hi, lo;
  split_tf32(v, hi, lo);
  Shi[o] = hi;
  Slo[o] = lo;
}

// Shared-memory matrix descriptor: no swizzle, K-major; lbo = byte distance of
// core matrices adjacent in K, sbo = of core matrices adjacent in M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, M x N.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's row (TMEM lane).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// C = X S for one 128 x kTN output tile (blockIdx.y: subdomain tile, blockIdx.x:
// boundary-dof tile), written to the copy slots of the interface dofs.  128
// threads: thread 0 streams the stages, thread 32 issues the MMAs, all four warps
// read the accumulator (warp w owns TMEM lanes 32w..32w+31 = output rows).
__global__ void __launch_bounds__(128, 1) k_schur_tc(DevMesh M, const int* __restrict__ sub_list, int n_list,
                                                     int n_bd, int nk, const float* __restrict__ Xhi,
                                                     const float* __restrict__ Xlo, const float* __restrict__ Shi,
                                                     const float* __restrict__ Slo, double* cbuf, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* s_fail = reinterpret_cast<int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nt = blockIdx.x, mt = blockIdx.y;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s]);
      mbar_init(&empty[s]);
    }
    mbar_init(done);
    *s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (threadIdx.x == 0) {
    // producer: stage ks % kStages, its u-th use waits for the MMAs of use u - 1
    int issued = 0;
    for (int ks = 0; ks < nk; ++ks) {
      const int st = ks % kStages, u = ks / kStages;
      if (u > 0 && !mbar_wait(&empty[st], (uint32_t)((u - 1) & 1))) {
        atomicOr(s_fail, 1);
        break;
      }
      unsigned char* base = smem + st * kStageBytes;
      mbar_expect_tx(&full[st], kStageBytes);
      const long long a_off = ((long long)mt * nk + ks) * (kTM * kTK);
      const long long b_off = ((long long)nt * nk + ks) * (kTN * kTK);
      bulk_copy_tx(base, Xhi + a_off, kABytes, &full[st]);
      bulk_copy_tx(base + kABytes, Xlo + a_off, kABytes, &full[st]);
      bulk_copy_tx(base + 2 * kABytes, Shi + b_off, kBBytes, &full[st]);
      bulk_copy_tx(base + 2 * kABytes + kBBytes, Slo + b_off, kBBytes, &full[st]);
      ++issued;
    }
    // every issued copy has landed before the CTA can leave (immediate on the normal path)
    for (int ks = issued - 1; ks >= 0 && ks >= issued - kStages; --ks)
      mbar_wait(&full[ks % kStages], (uint32_t)((ks / kStages) & 1));
  } else if (threadIdx.x == 32) {
    // MMA issuer
    for (int ks = 0; ks < nk; ++ks) {
      const int st = ks % kStages, u = ks / kStages;
      if (!mbar_wait(&full[st], (uint32_t)(u & 1))) {
        atomicOr(s_fail, 1);
        break;
      }
      tc_fence_after();
      const uint32_t a_hi = smem_addr(smem + st * kStageBytes), a_lo = a_hi + kABytes;
      const uint32_t b_hi = a_hi + 2 * kABytes, b_lo = b_hi + kBBytes;
#pragma unroll
      for (int s = 0; s < kTK / 8; ++s) {   // K = 8 per MMA: two core matrices along K
        const uint64_t dah = smem_desc(a_hi + s * 2 * (kTM / 8) * 128, (kTM / 8) * 128, 128);
        const uint64_t dal = smem_desc(a_lo + s * 2 * (kTM / 8) * 128, (kTM / 8) * 128, 128);
        const uint64_t dbh = smem_desc(b_hi + s * 2 * (kTN / 8) * 128, (kTN / 8) * 128, 128);
        const uint64_t dbl = smem_desc(b_lo + s * 2 * (kTN / 8) * 128, (kTN / 8) * 128, 128);
        mma_tf32(tmem, dah, dbh, (ks | s) != 0 ? 1u : 0u);
        mma_tf32(tmem, dah, dbl, 1u);
        mma_tf32(tmem, dal, dbh, 1u);
      }
      mma_commit(&empty[st]);   // stage free once these MMAs have read it
    }
    mma_commit(done);           // all MMAs issued by this thread complete
  }
  __syncwarp();
  if (!mbar_wait(done, 0u)) atomicOr(s_fail, 1);
  tc_fence_after();
  __syncthreads();
  const bool good = *s_fail == 0;   // the same for every thread: tcgen05.ld below is warp-collective
  if (good) {
    const int row = warp * 32 + lane;
    const int k = mt * kTM + row;
    for (int c0 = 0; c0 < kTN; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (k < n_list) {
        const SubDev& S = M.subs[sub_list[k]];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int i = nt * kTN + c0 + q;
          if (i < n_bd) {
            const int sl = M.sub_b2s[S.b2s_off + i / 3];
            if (sl >= 0) cbuf[(long long)sl + i % 3] = (double)v[q];
          }
        }
      }
    }
  }
  if (threadIdx.x == 0 && !good) atomicOr(err, 4);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

constexpr size_t kSmemTc = kStages * kStageBytes + (2 * kStages + 1) * sizeof(uint64_t) + 2 * sizeof(uint32_t);

}  // namespace

int schur_nk(int n_bd) { return (n_bd + kTK - 1) / kTK; }

long long schur_x_tile_floats(int n_list, int n_bd) {
  return (long long)((n_list + kTM - 1) / kTM) * kTM * schur_nk(n_bd) * kTK;
}

long long schur_s_tile_floats(int n_bd) {
  return (long long)((n_bd + kTN - 1) / kTN) * kTN * schur_nk(n_bd) * kTK;
}

void launch_schur_tile_S(const float* S32, int n_bd, float* Shi, float* Slo, cudaStream_t st) {
  const long long n = schur_s_tile_floats(n_bd);
  if (n > 0) k_schur_tile_S<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S32, n_bd, schur_nk(n_bd), Shi, Slo);
}

void launch_schur_gather(const DevMesh& M, const int* sub_list, int n_list, int n_bd, const double* lam, float* Xhi,
                         float* Xlo, cudaStream_t st) {
  const long long n = schur_x_tile_floats(n_list, n_bd);
  if (n > 0)
    k_schur_gather_tc<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M, sub_list, n_list, n_bd, schur_nk(n_bd), lam,
                                                                     Xhi, Xlo);
}

void launch_schur_gemm_scatter(const DevMesh& M, const int* sub_list, int n_list, int n_bd, const float* Xhi,
                               const float* Xlo, const float* Shi, const float* Slo, double* cbuf, int* err,
                               cudaStream_t st) {
  if (n_list <= 0 || n_bd <= 0) return;
  cudaFuncSetAttribute(k_schur_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTc);
  dim3 grid((unsigned)((n_bd + kTN - 1) / kTN), (unsigned)((n_list + kTM - 1) / kTM));
  k_schur_tc<<<grid, 128, kSmemTc, st>>>(M, sub_list, n_list, n_bd, schur_nk(n_bd), Xhi, Xlo, Shi, Slo, cbuf, err);
}

}  // namespace tfeti
