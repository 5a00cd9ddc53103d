// A6 / A10: tall-skinny Gram products G = A^T diag(w) B on the fifth-generation
// tensor cores (tcgen05), TF32 or BF16 inputs with FP32 accumulation, partial
// sums over row chunks added in FP64.
//
// A (n x M) and B (n x N) are column-major (each column contiguous): the
// reduction runs over the long dimension n, so both operands are "K-major".
// They are first packed into [cols][n_pad] buffers of the operand type (w
// folded into B, rows padded with zeros to a multiple of 64), which gives the
// tensor memory accelerator 16-byte-aligned rows.  Each CTA owns a 128 x NT
// tile of G and a contiguous range of 128-byte K slices: one thread streams
// the A and B boxes (128-byte swizzle) through a shared-memory ring of up to 8
// stages
// with cp.async.bulk.tensor, another issues tcgen05.mma into a TMEM
// accumulator (128 lanes x NT columns of FP32); tcgen05.commit releases each
// stage to the loader when the MMAs reading it complete.  The epilogue reads the accumulator with
// tcgen05.ld and writes the CTA's FP32 partial; a second kernel adds the
// partials of all K ranges in FP64 in a fixed order.  Every mbarrier wait is
// bounded: on a timeout the CTA sets the error flag, waits (bounded) for its
// MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>

#include "common.cuh"

namespace fdtdmor {

constexpr int TC_M = 128;        // rows of a G tile (TMEM lanes)
constexpr int TC_MAX_STAGES = 8;
constexpr int TC_ROWB = 128;     // bytes of K per row of a box (one swizzle row)
constexpr int TC_THREADS = 128;

__device__ __forceinline__ uint32_t tc_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tc_mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void tc_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_tma_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes in 8-row (1024-byte) groups; the group stride is 1024 bytes.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
  d |= (uint64_t)1 << 16;                      // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                      // descriptor version
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}

// Instruction descriptor: FP32 accumulator, A and B of format fmt (TF32 = 2
// for kind::tf32, BF16 = 1 for kind::f16), both K-major, M x N.
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <bool BF16>
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  if constexpr (BF16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// partial[z][m][n] (FP32) = sum over the K slices of range z of A[m][k] B[n][k]
// for the 128 x NT tile (blockIdx.x, blockIdx.y).  kslices: 128-byte K slices
// in all; per: slices per range.
template <bool BF16>
__global__ void __launch_bounds__(TC_THREADS, 1) gram_tc_kernel(const __grid_constant__ CUtensorMap ta,
                                                              const __grid_constant__ CUtensorMap tb, int M, int N,
                                                              int NT, int tmem_cols, int kslices, int per,
                                                              int TC_STAGES, float *__restrict__ partial,
                                                              unsigned *err) {
  extern __shared__ unsigned char tc_raw[];
  const uint32_t base = (tc_smem(tc_raw) + 1023u) & ~1023u;
  const uint32_t a_bytes = TC_M * TC_ROWB, b_bytes = (uint32_t)NT * TC_ROWB;
  const uint32_t stage_bytes = a_bytes + b_bytes;  // multiple of 1024 (NT a multiple of 16 -> 2 KB)
  const uint32_t bars = base + TC_STAGES * stage_bytes;  // full[S], empty[S], done
  const uint32_t full = bars, empty = bars + 8 * TC_STAGES, done = bars + 16 * TC_STAGES;
  const uint32_t tmem_slot = done + 8;
  unsigned char *slot_ptr = tc_raw + (tmem_slot - tc_smem(tc_raw));

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * TC_M, n0 = blockIdx.y * NT;
  const int ks0 = blockIdx.z * per, ks1 = min(kslices, ks0 + per);
  const int nk = max(0, ks1 - ks0);
  constexpr int KEL = TC_ROWB / (BF16 ? 2 : 4);   // elements per 128-byte slice
  constexpr uint32_t FMT = BF16 ? 1u : 2u;
  const uint32_t idesc = tc_idesc(FMT, TC_M, NT);

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      tc_mbar_init(full + 8 * s, 1);
      tc_mbar_init(empty + 8 * s, 1);
    }
    tc_mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tmem_slot), "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(slot_ptr);

  // warp 0 lane 0 streams the boxes, warp 1 lane 0 issues the MMAs
  bool ok = true;
  if (threadIdx.x == 0 && nk > 0) {
    for (int it = 0; it < nk; ++it) {
      const int s = it % TC_STAGES;
      if (it >= TC_STAGES && !tc_wait(empty + 8 * s, (uint32_t)((it / TC_STAGES) + 1) & 1u)) {
        ok = false;
        break;
      }
      const uint32_t sa = base + s * stage_bytes, sb = sa + a_bytes;
      tc_expect_tx(full + 8 * s, stage_bytes);
      const int kx = (ks0 + it) * KEL;
      tc_tma_2d(sa, &ta, kx, m0, full + 8 * s);
      tc_tma_2d(sb, &tb, kx, n0, full + 8 * s);
    }
    if (!ok) atomicOr(err, 4u);
  } else if (threadIdx.x == 32 && nk > 0) {
    for (int it = 0; it < nk; ++it) {
      const int s = it % TC_STAGES;
      if (!tc_wait(full + 8 * s, (uint32_t)(it / TC_STAGES) & 1u)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = base + s * stage_bytes, sb = sa + a_bytes;
#pragma unroll
      for (int kk = 0; kk < TC_ROWB / 32; ++kk)   // 32 bytes of K per MMA (8 TF32 / 16 BF16)
        tc_mma<BF16>(tmem, tc_desc(sa + 32 * kk), tc_desc(sb + 32 * kk), idesc, (it > 0 || kk > 0) ? 1u : 0u);
      tc_commit(empty + 8 * s);
    }
    tc_commit(done);   // also after a timeout: completes once the issued MMAs have
    if (!ok) atomicOr(err, 4u);
  }
  // epilogue: every thread owns one row of the tile
  const bool have = nk > 0 && tc_wait(done, 0);
  if (!have && nk > 0 && threadIdx.x == 0) atomicOr(err, 4u);
  ok = have;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int m = m0 + warp * 32 + lane;
  float *prow = partial + ((size_t)blockIdx.z * M + m) * N;
  for (int c = 0; c < NT; c += 8) {
    uint32_t r[8];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (m < M) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int n = n0 + c + q;
        if (n < N && c + q < NT) prow[n] = ok ? __uint_as_float(r[q]) : 0.0f;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
  }
}

// out[m][n] = sum_z partial[z][m][n] in FP64, fixed order.
__global__ void gram_tc_sum_kernel(int nsplit, int MN, const float *__restrict__ partial, double *__restrict__ out,
                                   int accumulate) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= MN) return;
  double a = 0;
  for (int z = 0; z < nsplit; ++z) a += (double)partial[(size_t)z * MN + t];
  out[t] = accumulate ? out[t] + a : a;
}

// Split of an FP32 operand into a head in the tensor-core input type and the
// remainder in the same type: v = hi + lo + O(2^-20 |v|) for TF32 (hi = v with
// the 13 low mantissa bits cleared, which is what the TF32 MMA reads of an
// FP32 value), O(2^-16 |v|) for BF16 (round to nearest twice).  Packed like
// gram_pack_kernel: dst[c][r], (w ? w[r] : 1) applied first, zeros past n.
template <typename D>
__global__ void gram_split_kernel(int64_t n, int64_t n_pad, const float *__restrict__ src, int64_t ld,
                                  const float *__restrict__ w, D *__restrict__ hi, D *__restrict__ lo) {
  const int c = blockIdx.y;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_pad; r += (int64_t)gridDim.x * blockDim.x) {
    float v = 0.0f;
    if (r < n) {
      v = src[(size_t)c * ld + r];
      if (w) v *= w[r];
    }
    const size_t o = (size_t)c * n_pad + r;
    if constexpr (sizeof(D) == 2) {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      hi[o] = h;
      lo[o] = __float2bfloat16_rn(v - __bfloat162float(h));
    } else {
      const float h = __uint_as_float(__float_as_uint(v) & 0xffffe000u);
      hi[o] = h;
      lo[o] = v - h;
    }
  }
}

// dst[c][r] = (w ? w[r] : 1) src[c * ld + r] for r < n, 0 for n <= r < n_pad.
template <typename D>
__global__ void gram_pack_kernel(int64_t n, int64_t n_pad, const float *__restrict__ src, int64_t ld,
                                 const float *__restrict__ w, D *__restrict__ dst) {
  const int c = blockIdx.y;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_pad; r += (int64_t)gridDim.x * blockDim.x) {
    float v = 0.0f;
    if (r < n) {
      v = src[(size_t)c * ld + r];
      if (w) v *= w[r];
    }
    if constexpr (sizeof(D) == 2) dst[(size_t)c * n_pad + r] = __float2bfloat16_rn(v);
    else dst[(size_t)c * n_pad + r] = v;
  }
}

typedef CUresult (*TcEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                               const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static TcEncodeFn tc_encode() {
  // looked up once (thread-safe static initialisation: batched builds call
  // this from several host threads)
  static const TcEncodeFn fn = []() -> TcEncodeFn {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<TcEncodeFn>(p);
    cudaGetLastError();
    return nullptr;
  }();
  return fn;
}

// 2-D map over a K-major operand of `rows` rows of n values (row stride ld
// values), box of 128 bytes x box_rows; reads past n or rows are zero.
static fdtd_status tc_map(CUtensorMap *m, bool bf16, void *base, int64_t n, int64_t ld, int rows, int box_rows) {
  TcEncodeFn fn = tc_encode();
  FDTD_REQUIRE(fn, "cuTensorMapEncodeTiled is not available");
  const int es = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * es};
  cuuint32_t box[2] = {(cuuint32_t)(TC_ROWB / es), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return FDTD_ECUDA;
  }
  return FDTD_OK;
}

// dst[c][r] (operand type, row stride n_pad) = (w ? w[r] : 1) src[c * ld + r]
// for r < n, 0 for n <= r < n_pad; c < ncols.
fdtd_status gram_pack(cudaStream_t s, bool bf16, int64_t n, int64_t n_pad, const float *src, int64_t ld, int ncols,
                      const float *w, void *dst) {
  if (ncols == 0) return FDTD_OK;
  FDTD_REQUIRE(ncols <= 65535, "gram_pack: at most 65535 columns");
  const int pbk = (int)std::min<int64_t>((n_pad + 255) / 256, 1024);
  if (bf16)
    gram_pack_kernel<__nv_bfloat16><<<dim3(pbk, ncols), 256, 0, s>>>(n, n_pad, src, ld, w,
                                                                     static_cast<__nv_bfloat16 *>(dst));
  else
    gram_pack_kernel<float><<<dim3(pbk, ncols), 256, 0, s>>>(n, n_pad, src, ld, w, static_cast<float *>(dst));
  return after_launch("gram_pack_kernel");
}

// G (M x N, row-major FP64) = A^T B for K-major operands already in the
// operand type: A rows (= columns of the original matrix) of n values with
// row stride lda, B likewise (strides x element size multiples of 16 bytes,
// 16-byte-aligned bases).  part: scratch for the FP32 partials.
fdtd_status gram_tensor_kmajor(cudaStream_t s, bool bf16, int64_t n, const void *A, int64_t lda, int M,
                               const void *B, int64_t ldb, int N, double *out, unsigned *err, DevBuf &part,
                               bool accumulate, int64_t max_rows) {
  if (M == 0 || N == 0) return FDTD_OK;
  const int es = bf16 ? 2 : 4;
  FDTD_REQUIRE(M <= 65535 && N <= 65535, "gram_tensor: at most 65535 columns");
  FDTD_REQUIRE((lda * es) % 16 == 0 && (ldb * es) % 16 == 0 && ((uintptr_t)A % 16) == 0 && ((uintptr_t)B % 16) == 0,
               "gram_tensor: operand rows must be 16-byte aligned");
  const int NT = std::min(256, (N + 15) / 16 * 16);
  int tmem_cols = 32;
  while (tmem_cols < NT) tmem_cols *= 2;
  const int mt = (M + TC_M - 1) / TC_M, ntl = (N + NT - 1) / NT;
  const int kslices = (int)((n * es + TC_ROWB - 1) / TC_ROWB);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int nsplit = std::max(1, std::min(kslices, std::max(1, sms) / std::max(1, mt * ntl)));  // one wave
  // at most max_rows rows per FP32 partial (their sum is FP64): a TMEM
  // accumulation over ~1e4 rows alone leaves ~1e-5 of relative error
  if (max_rows > 0) nsplit = std::max<int64_t>(nsplit, std::min<int64_t>(kslices, (n + max_rows - 1) / max_rows));
  const int per = (kslices + nsplit - 1) / nsplit;
  nsplit = (kslices + per - 1) / per;
  FDTD_CHECK(part.alloc((size_t)nsplit * M * N * sizeof(float), s));
  CUtensorMap ta, tb;
  FDTD_CHECK(tc_map(&ta, bf16, const_cast<void *>(A), n, lda, M, TC_M));
  FDTD_CHECK(tc_map(&tb, bf16, const_cast<void *>(B), n, ldb, N, NT));
  // as many stages as fit in 220 KB of shared memory
  const size_t stage = (size_t)(TC_M + NT) * TC_ROWB;
  const int nst = (int)std::max<size_t>(2, std::min<size_t>(TC_MAX_STAGES, (220 * 1024 - 1024 - 256) / stage));
  const size_t smem = 1024 + (size_t)nst * stage + 8 * (2 * nst + 1) + 16;
  auto kern = bf16 ? gram_tc_kernel<true> : gram_tc_kernel<false>;
  FDTD_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<dim3(mt, ntl, nsplit), TC_THREADS, smem, s>>>(ta, tb, M, N, NT, tmem_cols, kslices, per, nst, part.as<float>(),
                                                       err);
  FDTD_CHECK(after_launch("gram_tc_kernel"));
  const int MN = M * N;
  gram_tc_sum_kernel<<<(MN + 255) / 256, 256, 0, s>>>(nsplit, MN, part.as<float>(), out, accumulate ? 1 : 0);
  return after_launch("gram_tc_sum_kernel");
}

// G (M x N, row-major FP64) = A^T diag(w) B on the tensor cores; A: n x M with
// column stride lda, B: n x N with column stride ldb (FP32, device).
fdtd_status gram_tensor(cudaStream_t s, bool bf16, int64_t n, const float *A, int64_t lda, int M, const float *B,
                        int64_t ldb, int N, const float *w, double *out, unsigned *err) {
  if (M == 0 || N == 0) return FDTD_OK;
  const int64_t n_pad = std::max<int64_t>(64, (n + 63) / 64 * 64);
  const int es = bf16 ? 2 : 4;
  DevBuf pa, pb, part;
  struct Rel {
    DevBuf *a, *b, *c;
    cudaStream_t s;
    ~Rel() { a->release(s); b->release(s); c->release(s); }
  } rel{&pa, &pb, &part, s};
  // FP32 operands whose rows are already 16-byte aligned are read in place
  // (the tensor map zero-fills past n); others are packed once each
  auto aligned = [](const float *p, int64_t ld) { return (ld * 4) % 16 == 0 && ((uintptr_t)p % 16) == 0; };
  const void *pA = A, *pB = B;
  int64_t la = lda, lb = ldb, nk = n;
  const bool a_direct = !bf16 && aligned(A, lda), b_direct = !bf16 && !w && aligned(B, ldb);
  if (!(a_direct && b_direct)) {
    nk = n_pad;
    FDTD_CHECK(pa.alloc((size_t)M * n_pad * es, s));
    FDTD_CHECK(gram_pack(s, bf16, n, n_pad, A, lda, M, nullptr, pa.ptr));
    pA = pa.ptr;
    la = n_pad;
    if (B == A && ldb == lda && N == M && !w) {
      pB = pa.ptr;
    } else {
      FDTD_CHECK(pb.alloc((size_t)N * n_pad * es, s));
      FDTD_CHECK(gram_pack(s, bf16, n, n_pad, B, ldb, N, w, pb.ptr));
      pB = pb.ptr;
    }
    lb = n_pad;
  }
  return gram_tensor_kmajor(s, bf16, nk, pA, la, M, pB, lb, N, out, err, part, false, 0);
}

// Split-precision G = A^T diag(w) B on the tensor cores: with A = Ah + Al and
// B = Bh + Bl (gram_split_kernel), G = Ah^T Bh + Ah^T Bl + Al^T Bh in three
// tcgen05 passes, each with FP32 accumulation over row chunks and FP64 chunk
// sums; the dropped Al^T Bl and the split remainders are O(2^-20) of |A||B|
// for TF32 inputs, O(2^-16) for BF16.
// Rows per FP32 partial of the split-precision products (the partials are
// summed in FP64).  Measured on the 64^3 graded cavity with matched absorbers
// (q = 200, reduced-model probe error against the full-order run): 2048 rows
// 2.0e-3, 512 rows 3.4e-4 (FP32 CUDA-core products: 2.1e-4), 256 or 64 rows no
// better; the projection's time grows as the rows shrink (11, 15, 21, 64 ms).
constexpr int64_t kSplitRows = 512;

fdtd_status gram_tensor_split(cudaStream_t s, bool bf16, int64_t n, const float *A, int64_t lda, int M, const float *B,
                              int64_t ldb, int N, const float *w, double *out, unsigned *err) {
  if (M == 0 || N == 0) return FDTD_OK;
  FDTD_REQUIRE(M <= 65535 && N <= 65535, "gram_tensor_split: at most 65535 columns");
  const int64_t n_pad = std::max<int64_t>(64, (n + 63) / 64 * 64);
  const int es = bf16 ? 2 : 4;
  DevBuf ah, al, bh, bl, part;
  struct Rel {
    DevBuf *b[5];
    cudaStream_t s;
    ~Rel() { for (auto *x : b) x->release(s); }
  } rel{{&ah, &al, &bh, &bl, &part}, s};
  const int pbk = (int)std::min<int64_t>((n_pad + 255) / 256, 1024);
  auto split = [&](const float *src, int64_t ld, int ncols, const float *wt, DevBuf &h, DevBuf &l) -> fdtd_status {
    FDTD_CHECK(h.alloc((size_t)ncols * n_pad * es, s));
    FDTD_CHECK(l.alloc((size_t)ncols * n_pad * es, s));
    if (bf16)
      gram_split_kernel<__nv_bfloat16><<<dim3(pbk, ncols), 256, 0, s>>>(n, n_pad, src, ld, wt, h.as<__nv_bfloat16>(),
                                                                         l.as<__nv_bfloat16>());
    else
      gram_split_kernel<float><<<dim3(pbk, ncols), 256, 0, s>>>(n, n_pad, src, ld, wt, h.as<float>(), l.as<float>());
    return after_launch("gram_split_kernel");
  };
  FDTD_CHECK(split(A, lda, M, nullptr, ah, al));
  const bool same = B == A && ldb == lda && N == M && !w;
  if (!same) FDTD_CHECK(split(B, ldb, N, w, bh, bl));
  const void *Bh = same ? ah.ptr : bh.ptr, *Bl = same ? al.ptr : bl.ptr;
  const char *env = getenv("FDTDMOR_SPLIT_ROWS");
  const int64_t rows = env ? std::max<int64_t>(32, atoll(env)) : kSplitRows;
  FDTD_CHECK(gram_tensor_kmajor(s, bf16, n_pad, ah.ptr, n_pad, M, Bh, n_pad, N, out, err, part, false, rows));
  FDTD_CHECK(gram_tensor_kmajor(s, bf16, n_pad, ah.ptr, n_pad, M, Bl, n_pad, N, out, err, part, true, rows));
  return gram_tensor_kmajor(s, bf16, n_pad, al.ptr, n_pad, M, Bh, n_pad, N, out, err, part, true, rows);
}

}  // namespace fdtdmor
