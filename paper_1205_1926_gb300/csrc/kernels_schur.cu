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
// A second operand format stores S in BF16 (half the bytes of one FP32 copy):
// kind::f16 MMAs with BF16 operands and FP32 accumulation, X split into two BF16
// parts and D += X_hi S + X_lo S.  The product then carries S's BF16 rounding
// (~2^-9 relative); the FP64-refined PCGP around the inner solve absorbs it.
//
// Operand tiles are stored in global memory already in the shared-memory layout
// the MMA reads (no swizzle, K-major "core matrices" of 8 rows x 16 bytes), so
// one pipeline stage is a few contiguous 1-D bulk copies:
//   A (X) tile: 128 rows (subdomains) x 32 columns (dofs), core matrix (kg, mg)
//               at byte (kg * 16 + mg) * 128;  B (S) tile: kTN = 32 rows x 32 columns,
//               core matrix (kg, ng) at byte (kg * 4 + ng) * 128;
// row r of a core matrix holds 16 bytes of consecutive K elements (4 TF32 or 8 BF16).
#include <cuda_bf16.h>

#include "async_common.cuh"
#include "dev.h"
#include "dual_common.cuh"

namespace tfeti {

namespace {

constexpr int kTM = 128, kTN = 64, kTK = 32;
constexpr int kSU = 4;   // elements per thread of the scatter kernel, their loads in flight together
constexpr uint32_t kTmemCols = kTN;  // FP32 accumulator columns (a power of two >= 32)

// Operand format: TF32 x 3 (FP32 operands split into TF32 hi/lo, S hi/lo) or BF16 x 2
// (X split into BF16 hi/lo, S one BF16 copy).
template <bool kBf>
struct Fmt {
  static constexpr int eb = kBf ? 2 : 4;                       // bytes per element
  static constexpr int epr = 16 / eb;                          // elements per core-matrix row
  static constexpr int stages = kBf ? 8 : 4;
  static constexpr uint32_t a_bytes = kTM * kTK * eb, b_bytes = kTN * kTK * eb;
  static constexpr uint32_t stage_bytes = 2 * a_bytes + (kBf ? 1 : 2) * b_bytes;
  static constexpr int k_step = kBf ? 16 : 8;                  // K of one MMA
  // instruction descriptor: D FP32; A, B TF32 (kind::tf32) or BF16 (kind::f16); K-major; M x N
  static constexpr uint32_t idesc = (1u << 4) | ((kBf ? 1u : 2u) << 7) | ((kBf ? 1u : 2u) << 10) |
                                    ((uint32_t)(kTN >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
  static constexpr size_t smem = stages * stage_bytes + (2 * stages + 1) * sizeof(uint64_t) + 3 * sizeof(uint32_t);
};

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = tf32_round(x);
  lo = tf32_round(x - hi);
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Offset (elements) of element (row, col) inside an A tile (groups = 16) or a B tile
// (groups = 4), col < 32, for elements of epr per 16-byte core-matrix row.
__device__ __forceinline__ int tile_off(int row, int col, int groups, int epr) {
  return ((col / epr) * groups + (row >> 3)) * (8 * epr) + (row & 7) * epr + col % epr;
}

// X tiles: Xhi/Xlo[(mt * nk + ks) * 4096 + tile_off(r, c, 16)] for subdomain
// sub_list[mt * 128 + r] and boundary dof ks * 32 + c (zero beyond n_list, n_bd);
// elements TF32-split floats or BF16-split halves.
template <bool kBf>
__global__ void k_schur_gather_tc(DevMesh M, const int* __restrict__ sub_list, int n_list, int n_bd, int nk,
                                  const double* __restrict__ lam, void* Xhi, void* Xlo) {
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
  const long long o =
      ((long long)mt * nk + ks) * (kTM * kTK) + tile_off(k % kTM, j % kTK, kTM / 8, Fmt<kBf>::epr);
  if constexpr (kBf) {
    __nv_bfloat16 hi, lo;
    split_bf16(v, hi, lo);
    static_cast<__nv_bfloat16*>(Xhi)[o] = hi;
    static_cast<__nv_bfloat16*>(Xlo)[o] = lo;
  } else {
    float hi, lo;
    split_tf32(v, hi, lo);
    static_cast<float*>(Xhi)[o] = hi;
    static_cast<float*>(Xlo)[o] = lo;
  }
}

// cbuf at the interface slots of subdomain sub_list[k] = the sum over the K splits, in split
// order, of the GEMM's partial outputs part[z][k][i] (boundary dof i; row pitch n_nt * kTN).
// Consecutive threads take consecutive dofs of a subdomain (coalesced slot tables and stores);
// kSU elements per thread with their loads in flight together.
__global__ void k_schur_scatter(DevMesh M, const int* __restrict__ sub_list, int n_list, int n_bd, int n_mt, int n_nt,
                                int splits, const float* __restrict__ part, double* cbuf) {
  const long long ldp = (long long)n_nt * kTN, zs = (long long)n_mt * kTM * ldp;
  const long long n = (long long)n_list * n_bd, stride = (long long)gridDim.x * blockDim.x;
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < n; b += kSU * stride) {
    int k[kSU], i[kSU], sub[kSU];
#pragma unroll
    for (int u = 0; u < kSU; ++u) {
      const long long id = b + u * stride;
      k[u] = id < n ? (int)(id / n_bd) : -1;
      i[u] = id < n ? (int)(id % n_bd) : 0;
      sub[u] = k[u] >= 0 ? __ldg(sub_list + k[u]) : 0;
    }
    long long b2s[kSU];
    float v[kSU];
#pragma unroll
    for (int u = 0; u < kSU; ++u) {
      b2s[u] = k[u] >= 0 ? M.subs[sub[u]].b2s_off : 0;
      float acc = 0.f;
      if (k[u] >= 0) {
        const float* pk = part + (long long)k[u] * ldp + i[u];
        acc = __ldg(pk);
        for (int z = 1; z < splits; ++z) acc += __ldg(pk + z * zs);
      }
      v[u] = acc;
    }
    int sl[kSU];
#pragma unroll
    for (int u = 0; u < kSU; ++u) sl[u] = k[u] >= 0 ? __ldg(M.sub_b2s + b2s[u] + i[u] / 3) : -1;
#pragma unroll
    for (int u = 0; u < kSU; ++u)
      if (sl[u] >= 0) cbuf[(long long)sl[u] + i[u] % 3] = (double)v[u];
  }
}

// S tiles from the FP32 block S32 (S32[j * n_bd + i] = S[i][j]): TF32 hi/lo parts, or
// one BF16 copy (Slo unused).
template <bool kBf>
__global__ void k_schur_tile_S(const float* __restrict__ S32, int n_bd, int nk, void* Shi, void* Slo) {
  const long long ncol = (long long)nk * kTK;
  const int n_nt = (n_bd + kTN - 1) / kTN;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)n_nt * kTN * ncol) return;
  const int i = (int)(idx / ncol), j = (int)(idx % ncol);
  const float v = (i < n_bd && j < n_bd) ? S32[(long long)j * n_bd + i] : 0.0f;
  const int nt = i / kTN, ks = j / kTK;
  const long long o =
      ((long long)nt * nk + ks) * (kTN * kTK) + tile_off(i % kTN, j % kTK, kTN / 8, Fmt<kBf>::epr);
  if constexpr (kBf) {
    static_cast<__nv_bfloat16*>(Shi)[o] = __float2bfloat16_rn(v);
  } else {
    float hi, lo;
    split_tf32(v, hi, lo);
    static_cast<float*>(Shi)[o] = hi;
    static_cast<float*>(Slo)[o] = lo;
  }
}

// Shared-memory matrix descriptor: no swizzle, K-major; lbo = byte distance of
// core matrices adjacent in K, sbo = of core matrices adjacent in M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

template <bool kBf>
__device__ __forceinline__ void mma_issue(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  if constexpr (kBf) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(Fmt<true>::idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(Fmt<false>::idesc), "r"(accumulate)
        : "memory");
  }
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
// boundary-dof tile) over the K stages [ks0, ks1) of split blockIdx.z (gridDim.z > 1 when the
// output tiles alone would leave SMs idle), stored row-major in `part` for k_schur_scatter.
// 256 threads: thread 0 streams the stages, thread 32 issues the MMAs, and all eight warps
// read the accumulator: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its quadrant: output
// rows) and columns 32 (w / 4) .. + 31.  No CTA waits for another.
template <bool kBf>
__global__ void __launch_bounds__(256, 1) k_schur_tc(int nk, const unsigned char* __restrict__ Xhi,
                                                     const unsigned char* __restrict__ Xlo,
                                                     const unsigned char* __restrict__ Shi,
                                                     const unsigned char* __restrict__ Slo, float* part, int* err) {
  using F = Fmt<kBf>;
  constexpr int kSt = F::stages;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kSt * F::stage_bytes);
  uint64_t* empty = full + kSt;
  uint64_t* done = empty + kSt;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* s_flag = reinterpret_cast<int*>(tmem_slot + 1);   // [0]: a wait gave up
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nt = blockIdx.x, mt = blockIdx.y, splits = gridDim.z;
  const int ks0 = (int)((long long)blockIdx.z * nk / splits), ks1 = (int)((long long)(blockIdx.z + 1) * nk / splits);
  const int n_ks = ks1 - ks0;

  if (threadIdx.x == 0) {
    for (int q = 0; q < kSt; ++q) {
      mbar_init(&full[q]);
      mbar_init(&empty[q]);
    }
    mbar_init(done);
    s_flag[0] = 0;
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
    // producer: stage j % kSt, its u-th use waits for the MMAs of use u - 1
    int issued = 0;
    for (int j = 0; j < n_ks; ++j) {
      const int st = j % kSt, u = j / kSt, ks = ks0 + j;
      if (u > 0 && !mbar_wait(&empty[st], (uint32_t)((u - 1) & 1))) {
        atomicOr(&s_flag[0], 1);
        break;
      }
      unsigned char* base = smem + st * F::stage_bytes;
      mbar_expect_tx(&full[st], F::stage_bytes);
      const long long a_off = ((long long)mt * nk + ks) * F::a_bytes;
      const long long b_off = ((long long)nt * nk + ks) * F::b_bytes;
      bulk_copy_tx(base, Xhi + a_off, F::a_bytes, &full[st]);
      bulk_copy_tx(base + F::a_bytes, Xlo + a_off, F::a_bytes, &full[st]);
      bulk_copy_tx(base + 2 * F::a_bytes, Shi + b_off, F::b_bytes, &full[st]);
      if (!kBf) bulk_copy_tx(base + 2 * F::a_bytes + F::b_bytes, Slo + b_off, F::b_bytes, &full[st]);
      ++issued;
    }
    // every issued copy has landed before the CTA can leave (immediate on the normal path)
    for (int j = issued - 1; j >= 0 && j >= issued - kSt; --j)
      mbar_wait(&full[j % kSt], (uint32_t)((j / kSt) & 1));
  } else if (threadIdx.x == 32) {
    // MMA issuer: per stage, kTK / k_step MMA steps of two core matrices along K
    for (int j = 0; j < n_ks; ++j) {
      const int st = j % kSt, u = j / kSt;
      if (!mbar_wait(&full[st], (uint32_t)(u & 1))) {
        atomicOr(&s_flag[0], 1);
        break;
      }
      tc_fence_after();
      const uint32_t a_hi = smem_addr(smem + st * F::stage_bytes), a_lo = a_hi + F::a_bytes;
      const uint32_t b_hi = a_hi + 2 * F::a_bytes, b_lo = b_hi + F::b_bytes;
#pragma unroll
      for (int q = 0; q < kTK / F::k_step; ++q) {
        const uint64_t dah = smem_desc(a_hi + q * 2 * (kTM / 8) * 128, (kTM / 8) * 128, 128);
        const uint64_t dal = smem_desc(a_lo + q * 2 * (kTM / 8) * 128, (kTM / 8) * 128, 128);
        const uint64_t dbh = smem_desc(b_hi + q * 2 * (kTN / 8) * 128, (kTN / 8) * 128, 128);
        mma_issue<kBf>(tmem, dah, dbh, (j | q) != 0 ? 1u : 0u);
        if (!kBf) {
          const uint64_t dbl = smem_desc(b_lo + q * 2 * (kTN / 8) * 128, (kTN / 8) * 128, 128);
          mma_issue<kBf>(tmem, dah, dbl, 1u);
        }
        mma_issue<kBf>(tmem, dal, dbh, 1u);
      }
      mma_commit(&empty[st]);   // stage free once these MMAs have read it
    }
    mma_commit(done);           // all MMAs issued by this thread complete
  }
  __syncwarp();
  if (!mbar_wait(done, 0u)) atomicOr(&s_flag[0], 1);
  tc_fence_after();
  __syncthreads();
  const bool good = s_flag[0] == 0;   // the same for every thread: tcgen05.ld below is warp-collective
  // this split's output tile, row-major in part[split][m row][n column] (row pitch gridDim.x * kTN):
  // each lane holds one row of the accumulator and stores it as 16-float runs
  const int quad = warp & 3, cbeg = (warp >> 2) * (kTN / 2), cend = cbeg + kTN / 2;
  const int row = quad * 32 + lane;
  const long long ldp = (long long)gridDim.x * kTN;
  float* dst = part + (long long)blockIdx.z * ((long long)gridDim.y * kTM * ldp) + ((long long)mt * kTM + row) * ldp +
               (long long)nt * kTN;
  for (int c0 = cbeg; c0 < cend; c0 += 16) {
    float v[16];
    tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, v);
    float4* d4 = reinterpret_cast<float4*>(dst + c0);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      d4[q] = good ? make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (threadIdx.x == 0 && s_flag[0] != 0) atomicOr(err, 4);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace

int schur_nk(int n_bd) { return (n_bd + kTK - 1) / kTK; }

int schur_tiles(int n_list, int n_bd) { return ((n_list + kTM - 1) / kTM) * ((n_bd + kTN - 1) / kTN); }

long long schur_x_tile_elems(int n_list, int n_bd) {
  return (long long)((n_list + kTM - 1) / kTM) * kTM * schur_nk(n_bd) * kTK;
}

long long schur_s_tile_elems(int n_bd) {
  return (long long)((n_bd + kTN - 1) / kTN) * kTN * schur_nk(n_bd) * kTK;
}

long long schur_part_floats(int n_list, int n_bd, int splits) {
  return (long long)schur_tiles(n_list, n_bd) * splits * kTM * kTN;
}

void launch_schur_tile_S(const float* S32, int n_bd, bool bf16, void* Shi, void* Slo, cudaStream_t st) {
  const long long n = schur_s_tile_elems(n_bd);
  if (n <= 0) return;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (bf16) k_schur_tile_S<true><<<blocks, 256, 0, st>>>(S32, n_bd, schur_nk(n_bd), Shi, Slo);
  else k_schur_tile_S<false><<<blocks, 256, 0, st>>>(S32, n_bd, schur_nk(n_bd), Shi, Slo);
}

void launch_schur_gather(const DevMesh& M, const int* sub_list, int n_list, int n_bd, bool bf16, const double* lam,
                         void* Xhi, void* Xlo, cudaStream_t st) {
  const long long n = schur_x_tile_elems(n_list, n_bd);
  if (n <= 0) return;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (bf16) k_schur_gather_tc<true><<<blocks, 256, 0, st>>>(M, sub_list, n_list, n_bd, schur_nk(n_bd), lam, Xhi, Xlo);
  else k_schur_gather_tc<false><<<blocks, 256, 0, st>>>(M, sub_list, n_list, n_bd, schur_nk(n_bd), lam, Xhi, Xlo);
}

int schur_splits(int n_list, int n_bd, int n_sm) {
  // two splits of K when the output tiles alone would leave SMs idle (and K is long enough)
  return (schur_tiles(n_list, n_bd) < n_sm && schur_nk(n_bd) >= 8) ? 2 : 1;
}

void launch_schur_gemm_scatter(const DevMesh& M, const int* sub_list, int n_list, int n_bd, bool bf16, int splits,
                               const void* Xhi, const void* Xlo, const void* Shi, const void* Slo, float* part,
                               double* cbuf, int* err, cudaStream_t st) {
  if (n_list <= 0 || n_bd <= 0) return;
  const int n_nt = (n_bd + kTN - 1) / kTN, n_mt = (n_list + kTM - 1) / kTM;
  dim3 grid((unsigned)n_nt, (unsigned)n_mt, (unsigned)splits);
  const auto* xh = static_cast<const unsigned char*>(Xhi);
  const auto* xl = static_cast<const unsigned char*>(Xlo);
  const auto* sh = static_cast<const unsigned char*>(Shi);
  const auto* sl = static_cast<const unsigned char*>(Slo);
  if (bf16) {
    cudaFuncSetAttribute(k_schur_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Fmt<true>::smem);
    k_schur_tc<true><<<grid, 256, Fmt<true>::smem, st>>>(schur_nk(n_bd), xh, xl, sh, sl, part, err);
  } else {
    cudaFuncSetAttribute(k_schur_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Fmt<false>::smem);
    k_schur_tc<false><<<grid, 256, Fmt<false>::smem, st>>>(schur_nk(n_bd), xh, xl, sh, sl, part, err);
  }
  const long long n = (long long)n_list * n_bd;
  const unsigned blocks = (unsigned)((n + 256LL * kSU - 1) / (256LL * kSU));
  k_schur_scatter<<<blocks, 256, 0, st>>>(M, sub_list, n_list, n_bd, n_mt, n_nt, splits, part, cbuf);
}

}  // namespace tfeti
