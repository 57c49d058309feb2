// FP32-accurate GEMM on the tcgen05 tensor cores (3xTF32).
//
//   D[m, n] = sum_k A[m, k] B[n, k]         (A: M x K, B: N x K, both K-major)
//
// Each FP32 operand x is given as a TF32 pair x = hi + lo (hi = x rounded to
// TF32, lo = x - hi, exact in FP32); the product keeps hi*hi + hi*lo + lo*hi
// and drops lo*lo (relative 2^-22), so the result is within a few FP32 ulps
// of an FP32 GEMM while running on the tensor pipe.  The dense contractions
// of the FP32 local operator (rank >= 32) use it.
//
// One 128 x 128 output tile per CTA of 128 threads:
//   * thread 0 loads 32-deep K slices of A_hi, A_lo, B_hi, B_lo with TMA
//     (128-byte swizzle) into a three-stage ring guarded by mbarriers;
//   * thread 32 issues the MMAs (three per 8-deep step) into a 128 x 128
//     FP32 accumulator in tensor memory and releases each stage with
//     tcgen05.commit;
//   * all four warps read the accumulator back (tcgen05.ld, warp w owns
//     lanes 32w..32w+31 = rows) and store it through an index map, either
//     as FP32 or again as a TF32 hi/lo pair for the next contraction.
// Every wait on an mbarrier is bounded; a wait that gives up records
// QTT_ETIMEOUT in the error word and the CTA skips to its clean-up.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace qtt {
namespace {

constexpr int BM = 128, BN = 128, BK = 32, STAGES = 3;
constexpr int TILE_BYTES = BM * BK * 4;          // 16 KB (BN == BM)
constexpr int STAGE_BYTES = 4 * TILE_BYTES;      // A_hi, A_lo, B_hi, B_lo
constexpr int BAR_BYTES = 256;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + BAR_BYTES + 1024;   // + alignment slack
constexpr long long WAIT_LIMIT = 1LL << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile whose rows are 128-byte
// lines in the 128-byte swizzle pattern (as TMA writes them): 8-row groups
// 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);          // start address, 16-byte units
  d |= (uint64_t)1 << 16;                           // leading-dimension offset (unused when swizzled)
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride between 8-row groups
  d |= (uint64_t)1 << 46;                           // descriptor version of tcgen05
  d |= (uint64_t)2 << 61;                           // 128-byte swizzle
  return d;
}

// Instruction descriptor: kind::tf32, FP32 accumulator, A and B TF32 and
// K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ long long map_off(const TcIdxMap& d, int idx) {
  long long o = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (t < d.cnt) {
      o += (long long)(idx % d.n[t]) * d.s[t];
      idx /= d.n[t];
    }
  }
  return o;
}

__global__ void __launch_bounds__(128, 1)
    tf32x3_gemm_kernel(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                       const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl, int M, int N,
                       int K, int kb_per, TcEpilogue epi, int* err) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;                 // 1024-byte aligned tiles
  const uint32_t bars = base + STAGES * STAGE_BYTES;            // full[S], empty[S], done, tmem slot
  unsigned char* gbase = smem_raw + (base - raw);
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(gbase + STAGES * STAGE_BYTES + 8 * (2 * STAGES + 1));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kb0 = blockIdx.z * kb_per;                        // this split's K slices
  const int nk = min((K + BK - 1) / BK - kb0, kb_per);
  auto full = [&](int st) { return bars + 8u * st; };
  auto empty = [&](int st) { return bars + 8u * (STAGES + st); };
  const uint32_t done = bars + 8u * (2 * STAGES);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(const_cast<uint32_t*>(tmem_slot))),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int st = 0; st < STAGES; ++st) {
      mbar_init(full(st), 1);
      mbar_init(empty(st), 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (threadIdx.x == 0) {
    // producer: K slices into the ring
    int issued = 0;
    for (int kb = 0; kb < nk && ok; ++kb) {
      const int st = kb % STAGES;
      if (kb >= STAGES) ok = mbar_wait(empty(st), (uint32_t)((kb / STAGES - 1) & 1));
      if (!ok) break;
      const uint32_t sb = base + st * STAGE_BYTES;
      mbar_expect_tx(full(st), STAGE_BYTES);
      const int kx = (kb0 + kb) * BK;
      tma_load_2d(sb, &tAh, full(st), kx, m0);
      tma_load_2d(sb + TILE_BYTES, &tAl, full(st), kx, m0);
      tma_load_2d(sb + 2 * TILE_BYTES, &tBh, full(st), kx, n0);
      tma_load_2d(sb + 3 * TILE_BYTES, &tBl, full(st), kx, n0);
      issued = kb + 1;
    }
    // no copy may still be landing in shared memory when the CTA leaves
    // (returns at once when the MMA thread has consumed every stage)
    for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
      if (!mbar_wait(full(kb % STAGES), (uint32_t)((kb / STAGES) & 1))) ok = false;
    if (!ok) atomicExch(err, QTT_ETIMEOUT);
  } else if (threadIdx.x == 32) {
    // MMA issuer
    const uint32_t idesc = idesc_tf32(BM, BN);
    for (int kb = 0; kb < nk && ok; ++kb) {
      const int st = kb % STAGES;
      ok = mbar_wait(full(st), (uint32_t)((kb / STAGES) & 1));
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sb = base + st * STAGE_BYTES;
#pragma unroll
      for (int ks = 0; ks < BK / 8; ++ks) {        // 8 TF32 = 32 bytes per MMA step
        const uint32_t off = ks * 32;
        const uint64_t ah = desc_sw128(sb + off), al = desc_sw128(sb + TILE_BYTES + off);
        const uint64_t bh = desc_sw128(sb + 2 * TILE_BYTES + off), bl = desc_sw128(sb + 3 * TILE_BYTES + off);
        mma_tf32(tmem, ah, bh, idesc, (kb > 0 || ks > 0) ? 1u : 0u);
        mma_tf32(tmem, ah, bl, idesc, 1u);
        mma_tf32(tmem, al, bh, idesc, 1u);
      }
      mma_commit(empty(st));                       // the stage is free once these MMAs are done
    }
    // `done` arrives once every MMA issued so far has completed, also after
    // a timeout, so that tensor memory is never released under them
    mma_commit(done);
    if (!ok) atomicExch(err, QTT_ETIMEOUT);
  }
  __syncwarp();
  // epilogue: every thread owns one row of the tile
  bool have = mbar_wait(done, 0);
  if (!have && lane == 0) atomicExch(err, QTT_ETIMEOUT);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (have && __all_sync(0xffffffffu, have)) {
    const int m = m0 + warp * 32 + lane;
    const long long om = (m < M) ? map_off(epi.om, m) : 0;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int n = n0 + c0 + j;
        if (n >= N) break;
        const long long o = om + map_off(epi.on, n);
        const float v = __uint_as_float(r[j]);
        if (epi.lo) {
          const float h = tf32_round(v);
          epi.out[o] = h;
          epi.lo[o] = v - h;
        } else if (epi.atomic) {
          atomicAdd(epi.out + o, v);
        } else {
          epi.out[o] = v;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

__global__ void tf32_split_kernel(const float* __restrict__ x, float* __restrict__ hi, float* __restrict__ lo,
                                  long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float v = x[i];
    const float h = tf32_round(v);
    hi[i] = h;
    lo[i] = v - h;
  }
}

// hi/lo TF32 pairs of a rows x K K-major operand gathered from a tensor:
// element (row, k) = src[rmap(row) + kmap(k)].  32 x 32 tiles through shared
// memory: reads run along rows, writes along k.
__global__ void __launch_bounds__(256) pack_pairs_kernel(const float* __restrict__ src, int rows, int K, int ld,
                                                         TcIdxMap rmap, TcIdxMap kmap, float* __restrict__ hi,
                                                         float* __restrict__ lo) {
  __shared__ float tile[32][33];
  const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int kk = threadIdx.y; kk < 32; kk += 8) {
    const int r = r0 + threadIdx.x, k = k0 + kk;
    tile[kk][threadIdx.x] = (r < rows && k < K) ? src[map_off(rmap, r) + map_off(kmap, k)] : 0.f;
  }
  __syncthreads();
  for (int rr = threadIdx.y; rr < 32; rr += 8) {
    const int r = r0 + rr, k = k0 + threadIdx.x;
    if (r < rows && k < K) {
      const float v = tile[threadIdx.x][rr];
      const float h = tf32_round(v);
      hi[(size_t)r * ld + k] = h;
      lo[(size_t)r * ld + k] = v - h;
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

// rows x K matrix, K-major with leading dimension ld (elements), box 32 x 128
CUtensorMap make_map(const float* p, int rows, int K, int ld) {
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {BK, BM};
  const cuuint32_t estr[2] = {1, 1};
  auto fn = encode_fn();
  QTT_REQUIRE(fn, "tf32x3 gemm: cuTensorMapEncodeTiled is not available");
  CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(p), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw QttError(QTT_ECUDA, "tf32x3 gemm: tensor map encoding failed (" + std::to_string((int)r) + ")");
  return m;
}

}  // namespace

bool tc_available() {
  static int ok = -1;
  if (ok < 0) {
    int dev = 0, major = 0, minor = 0;
    ok = (cudaGetDevice(&dev) == cudaSuccess &&
          cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) == cudaSuccess &&
          cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) == cudaSuccess && major == 10 &&
          minor == 3 && encode_fn() != nullptr)
             ? 1
             : 0;
    cudaGetLastError();
  }
  return ok == 1;
}

void tc_pack(cudaStream_t s, const float* src, int rows, int K, int ld, const TcIdxMap& rmap, const TcIdxMap& kmap,
             float* hi, float* lo) {
  if (rows <= 0 || K <= 0) return;
  QTT_REQUIRE((K + 31) / 32 <= 65535, "tc_pack: K too large");
  dim3 grid((rows + 31) / 32, (K + 31) / 32);
  pack_pairs_kernel<<<grid, dim3(32, 8), 0, s>>>(src, rows, K, ld, rmap, kmap, hi, lo);
  QTT_CHECK_LAUNCH();
}

void tf32_split(cudaStream_t s, const float* x, float* hi, float* lo, long long n) {
  if (n <= 0) return;
  tf32_split_kernel<<<grid_for_n(n, 8), 256, 0, s>>>(x, hi, lo, n);
  QTT_CHECK_LAUNCH();
}

void tc_plan(TcGemmPlan& p, int M, int N, int K, const float* Ahi, const float* Alo, int lda, const float* Bhi,
             const float* Blo, int ldb, const TcEpilogue& epi, int max_splits) {
  QTT_REQUIRE(M >= 1 && N >= 1 && K >= 1, "tf32x3 gemm: sizes must be positive");
  QTT_REQUIRE(lda % 4 == 0 && ldb % 4 == 0 && lda >= K && ldb >= K,
              "tf32x3 gemm: leading dimensions must be multiples of 4 elements (16-byte TMA strides)");
  auto aligned16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
  QTT_REQUIRE(aligned16(Ahi) && aligned16(Alo) && aligned16(Bhi) && aligned16(Blo),
              "tf32x3 gemm: operands must start on 16-byte boundaries");
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  const CUtensorMap maps[4] = {make_map(Ahi, M, K, lda), make_map(Alo, M, K, lda), make_map(Bhi, N, K, ldb),
                               make_map(Blo, N, K, ldb)};
  std::memcpy(p.maps, maps, sizeof(maps));
  p.M = M;
  p.N = N;
  p.K = K;
  const int nk = (K + BK - 1) / BK;
  int splits = std::max(1, std::min(max_splits, nk));
  if (epi.lo || !epi.atomic) splits = 1;
  p.kb_per = (nk + splits - 1) / splits;
  p.splits = (nk + p.kb_per - 1) / p.kb_per;       // every split has at least one K slice
  p.epi = epi;
  QTT_REQUIRE((M + BM - 1) / BM <= 2147483647 && (N + BN - 1) / BN <= 65535 && p.splits <= 65535,
              "tf32x3 gemm: grid too large");
}

void tc_run(cudaStream_t s, const TcGemmPlan& p, int* err) {
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(tf32x3_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  });
  const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(p.maps);
  dim3 grid((p.M + BM - 1) / BM, (p.N + BN - 1) / BN, p.splits);
  ProfToken pt = prof_begin(PROF_TC_GEMM, s);
  tf32x3_gemm_kernel<<<grid, 128, SMEM_BYTES, s>>>(m[0], m[1], m[2], m[3], p.M, p.N, p.K, p.kb_per, p.epi, err);
  QTT_CHECK_LAUNCH();
  if (pt.ev)
    prof_end(pt, s, 2.0 * p.M * p.N * p.K,
             4.0 * (2.0 * p.M * p.K + 2.0 * p.N * p.K + (p.epi.lo ? 2.0 : 1.0) * p.M * p.N));
}

void tf32x3_gemm(cudaStream_t s, int M, int N, int K, const float* Ahi, const float* Alo, int lda, const float* Bhi,
                 const float* Blo, int ldb, const TcEpilogue& epi, int* err) {
  if (M <= 0 || N <= 0) return;
  TcGemmPlan p;
  tc_plan(p, M, N, K, Ahi, Alo, lda, Bhi, Blo, ldb, epi, 1);
  tc_run(s, p, err);
}

}  // namespace qtt

extern "C" int qtt_gemm_tf32x3(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* D,
                               int ldd, void* stream) {
  try {
    QTT_REQUIRE(A && B && D, "qtt_gemm_tf32x3: null argument");
    QTT_REQUIRE(M >= 0 && N >= 0 && K >= 1 && lda >= K && ldb >= K && ldd >= std::max(1, M),
                "qtt_gemm_tf32x3: bad sizes or leading dimensions");
    QTT_REQUIRE(qtt::tc_available(), "qtt_gemm_tf32x3: needs an sm_103 device (tcgen05)");
    if (M == 0 || N == 0) return QTT_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    qtt::StreamScope scope_(s);
    qtt::Arena ar(s);
    const int ldk = (K + 3) / 4 * 4;
    float* tmp = ar.alloc<float>((size_t)std::max(M, N) * ldk);
    float* Ah = ar.alloc<float>((size_t)M * ldk);
    float* Al = ar.alloc<float>((size_t)M * ldk);
    float* Bh = ar.alloc<float>((size_t)N * ldk);
    float* Bl = ar.alloc<float>((size_t)N * ldk);
    int* err = ar.alloc<int>(1);
    QTT_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    // K-major copies with a 16-byte-multiple leading dimension (zero padding)
    QTT_CUDA(cudaMemsetAsync(tmp, 0, sizeof(float) * (size_t)std::max(M, N) * ldk, s));
    qtt::copy2d<float>(s, K, M, A, lda, tmp, ldk);
    qtt::tf32_split(s, tmp, Ah, Al, (long long)M * ldk);
    qtt::copy2d<float>(s, K, N, B, ldb, tmp, ldk);
    qtt::tf32_split(s, tmp, Bh, Bl, (long long)N * ldk);
    qtt::TcEpilogue epi{};
    epi.om.cnt = 1;
    epi.om.n[0] = M;
    epi.om.s[0] = 1;
    epi.on.cnt = 1;
    epi.on.n[0] = N;
    epi.on.s[0] = ldd;
    epi.out = D;
    epi.lo = nullptr;
    // too few output tiles to fill the SMs: split K, accumulate atomically
    const long long tiles = (long long)((M + 127) / 128) * ((N + 127) / 128);
    const int want = (int)std::max<long long>(1, (2LL * qtt::num_sms() + tiles - 1) / tiles);
    epi.atomic = want > 1 ? 1 : 0;
    if (epi.atomic) QTT_CUDA(cudaMemset2DAsync(D, sizeof(float) * (size_t)ldd, 0, sizeof(float) * (size_t)M, N, s));
    qtt::TcGemmPlan plan;
    qtt::tc_plan(plan, M, N, K, Ah, Al, ldk, Bh, Bl, ldk, epi, want);
    qtt::tc_run(s, plan, err);
    int herr = 0;
    QTT_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    QTT_CUDA(cudaStreamSynchronize(s));
    if (herr != 0) throw qtt::QttError(herr, "qtt_gemm_tf32x3: a bounded wait in the kernel gave up");
    return QTT_OK;
  } catch (const qtt::QttError& e) {
    qtt::set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    qtt::set_last_error(e.what());
    return QTT_EINVAL;
  }
}
