// contract_tc.cu -- the blend-accumulate walk (Eq. 4-6) with its per-tile contraction on the
// 5th-generation tensor cores (tcgen05), for 16-bit targets with 16..64 channels.
//
// Per tile and batch of MG = 64 Gaussians (the MMA's M; 64 rather than 128 halves the weight
// operand, so that 3-5 CTAs fit on an SM), the S terms of Eq. 6 summed over the tile's 256 pixels
// form a dense product
//     D[g][n] = sum_p W[g][p] * B[n][p],   W[g][p] = alpha T of Gaussian g at pixel p (Eq. 4),
// with B's rows 0..KT-1 the tile's target channels and the rows after them all ones, so that the same
// product also yields V = sum_p W[g][p] (Eq. 5). The threads evaluate W with the same decisions as
// the CUDA-core walks (walk.cuh: branch-free, two hits a step) and store it as FP16 into a K-major,
// 128-byte-swizzled shared-memory operand; the tile's targets (BF16 or FP16) are transposed once
// into B as FP16. Both operands are scaled by powers of two -- W by 2^14 (the walk carries T scaled
// so), the targets so that the tile's largest magnitude lands in [2^14, 2^15) -- which makes every
// BF16 target exact in FP16, keeps small weights out of FP16's subnormal range, and is undone exactly
// in the epilogue. One thread issues 16 tcgen05.mma (kind::f16, M=MG, N=KT+8, K=16, FP32
// accumulation in TMEM) and commits them to an mbarrier; while they run, the next batch's Gaussians
// are staged (the geometry into the buffer the walk has finished with, each index into the register
// of the thread that adds its row); the warps then read D back with tcgen05.ld (one Gaussian per
// thread, the chunks split between warps w and w+4) and add (V, S_0..S_{KT-1}) to the accumulator
// with float4 atomics -- one atomic group per (Gaussian, tile). A batch costs two CTA barriers. At 16
// channels the whole layout takes 44 KiB (five CTAs per SM): see b16_offset and tc_smem.
//
// Every wait on the mbarrier is bounded in time (1 s by %globaltimer): past the limit the kernel
// sets kFlagTimeout in the status block (reported as ICGS_ERR_DEVICE_TIMEOUT), waits once more
// (also bounded) for the MMAs it issued, frees its TMEM and returns. A diagnostic entry point
// (icgs_debug_tc_wait) shortens the limit and can leave the MMAs unissued, so that a test drives a
// wait past its limit with nothing in flight.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "icgs_device.cuh"
#include "icgs_internal.h"
#include "walk.cuh"

namespace icgs {

namespace {

using namespace walk;

constexpr int kG = 128;                 // rows of the self-test MMA (the walk uses MG = 64)
constexpr int kKPix = 256;              // pixels per tile (MMA K in total, 16 instructions of 16)
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // bounded mbarrier waits give up after 1 s
constexpr uint32_t kTmemCols = 128;     // TMEM columns of the self-test (N <= 80)

// ---- inline PTX ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait; returns false (and the caller reports a timeout) once limit_ns have passed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs) {
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(mbar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}

// D[tmem] (+)= A[smem] * B[smem]^T, both operands K-major, kind::f16 (BF16 or FP16 in, FP32 out)
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on the mbarrier once every MMA this thread issued has completed.
__device__ __forceinline__ void umma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}
// 16 consecutive 32-bit columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---- operand layout -------------------------------------------------------------------------
// A [rows x 256] 16-bit matrix stored K-major with the 128-byte swizzle: four K blocks of 64
// elements, each block rows x 128 bytes, rows grouped by 8 into 1024-byte atoms, and the 16-byte
// chunk index of each row XOR-ed with the row's index inside its atom.
__device__ __forceinline__ uint32_t kmajor_sw128(int row, int k, int rows) {
  return (uint32_t)((k >> 6) * (rows * 128) + (row >> 3) * 1024 + (row & 7) * 128 +
                    ((((k & 63) >> 3) ^ (row & 7)) << 4) + ((k & 7) << 1));
}

// Shared-memory matrix descriptor (tcgen05 format): start address >> 4 in bits 0-13, leading byte
// offset >> 4 in bits 16-29 (unused for swizzled K-major; 1 by convention), stride byte offset
// >> 4 in bits 32-45 (1024 B between 8-row atoms), descriptor version 1 in bits 46-47, layout type
// in bits 61-63 (2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t desc_kmajor_sw128(uint32_t saddr, uint32_t sbo = 1024) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(sbo >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: D format F32 (bits 4-5 = 1), A and B format (bits 7-9,
// 10-12: 0 = F16, 1 = BF16), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in
// bits 24-28.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, bool bf16) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

constexpr int kWScaleExp = 14;  // W is stored as W * 2^14 (W < 1)

__device__ __forceinline__ uint16_t half_bits(float x) { return __half_as_ushort(__float2half_rn(x)); }
__device__ __forceinline__ float target_value(uint16_t raw, bool bf16) {
  return bf16 ? __uint_as_float((uint32_t)raw << 16) : __half2float(__ushort_as_half(raw));
}

// Issues the 16 MMAs of one batch (K = 256 pixels) and commits them to mbar.
template <int NB, int MG = kG>
__device__ __forceinline__ void issue_batch(uint32_t a_addr, uint32_t b_addr, uint32_t d_tmem, uint32_t idesc,
                                            uint64_t* mbar) {
  tc_fence_after();
#pragma unroll
  for (int ks = 0; ks < kKPix / 16; ++ks) {
    const int kb = ks >> 2, kk = ks & 3;
    const uint64_t ad = desc_kmajor_sw128(a_addr + kb * (MG * 128) + kk * 32);
    const uint64_t bd = desc_kmajor_sw128(b_addr + kb * (NB * 128) + kk * 32);
    umma_f16(d_tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
  }
  umma_commit(mbar);
}

// ---- B of the 16-channel walk in 11 KB ---------------------------------------------------------
// B is [24 x 256]: 16 target rows (two 8-row atoms per K block of 64 pixels) and 8 rows of ones. An
// MMA reads its three atoms at start, start + SBO and start + 2 SBO, and every MMA has its own
// descriptor, so each K block kb gets its own stride s_kb (in KB) and puts its two target atoms at
// 2 s_kb and s_kb KB below one shared atom of ones. With s = 1, 3, 4, 5 the eight target atoms and
// the ones occupy KB 0, 2, 4-10 of an 11 KB region (ones at KB 10); KB 1 and 3 hold the staged
// geometry. The ones' values do not depend on the pixel, so every K block may read the same atom.
__host__ __device__ constexpr int b16_stride_kb(int kb) { return kb == 0 ? 1 : kb + 2; }
constexpr uint32_t kB16Ones = 10 * 1024;  // offset of the ones atom in the region
constexpr uint32_t kB16Bytes = 11 * 1024;
constexpr uint32_t kB16Geo = 1 * 1024, kB16Aux = 3 * 1024;  // the holes

// byte offset of B[channel k][pixel p] (k < 16) in the region
__device__ __forceinline__ uint32_t b16_offset(int k, int p) {
  const int kb = p >> 6, s = b16_stride_kb(kb);
  const uint32_t atom = kB16Ones - (uint32_t)((k < 8 ? 2 : 1) * s) * 1024u;
  return atom + (uint32_t)((k & 7) * 128 + ((((p & 63) >> 3) ^ (k & 7)) << 4) + ((p & 7) << 1));
}

// The 16 MMAs of one batch of the 16-channel walk (N = 24: columns 0-15 the targets, 16-23 V).
template <int MG>
__device__ __forceinline__ void issue_batch_b16(uint32_t a_addr, uint32_t b_region, uint32_t d_tmem, uint32_t idesc,
                                                uint64_t* mbar) {
  tc_fence_after();
#pragma unroll
  for (int ks = 0; ks < kKPix / 16; ++ks) {
    const int kb = ks >> 2, kk = ks & 3, sk = b16_stride_kb(kb);
    const uint64_t ad = desc_kmajor_sw128(a_addr + kb * (MG * 128) + kk * 32);
    const uint64_t bd = desc_kmajor_sw128(b_region + kB16Ones - (uint32_t)(2 * sk) * 1024u + kk * 32, (uint32_t)sk * 1024u);
    umma_f16(d_tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
  }
  umma_commit(mbar);
}

// Staging of a batch for the walk (M = 64). The thread that stages Gaussian g is the one that adds
// row g's sums in the epilogue -- lane g % 16 of warp g / 16, since TMEM holds row g in lane g % 16
// of quarter g / 16 -- so the Gaussian's index stays in that thread's register from staging to
// epilogue. Warps 4-7 read the same quarters for the later accumulator columns (more than 16
// channels); their lanes < 16 load only the index (need_id).
__device__ __forceinline__ uint32_t stage_tc(const unsigned long long* list, uint32_t first, int nb,
                                             const ProjRec* __restrict__ rec_cam, int64_t n, float ox, float oy,
                                             float4* s_geo, float4* s_aux, int g, bool writer, bool need_id) {
  uint32_t id = 0;
  if (g >= 0 && g < nb && (writer || need_id)) {
    id = min((uint32_t)list[first + g], (uint32_t)(n - 1));
    if (writer) {
      // aux = (C, opacity, the slot's row offset in W, packed half-sizes): the walk's step needs no
      // fast-reject threshold (blend_alpha_noreject), so the third value carries g * 128 +
      // (g % 8) * 16, the Gaussian's part of its weights' swizzled address
      const ProjRec r = rec_cam[id];
      s_geo[g] = stage_geo(r, ox, oy);
      s_aux[g] = make_float4(-kHalfLog2e * r.par.z, r.par.w, __uint_as_float((uint32_t)((g << 7) | ((g & 7) << 4))),
                             r.box.w);
    }
  }
  return id;
}

// The accumulator row held in TMEM lane 32 q + l (the lane a thread l of a warp with quarter q
// reads), or -1: M = 128 puts row m in lane m; M = 64 puts row m in lane (m % 16) + 32 (m / 16),
// i.e. rows 16q..16q+15 in the first 16 lanes of quarter q.
template <int MG>
__device__ __forceinline__ int tmem_row_of_lane(int q, int l) {
  return MG == 128 ? q * 32 + l : (l < 16 ? q * 16 + l : -1);
}

// ---- self-test: D[M x N] = A[M x 256] B[N x 256]^T through the same layout and MMA path ----
// (M = 64 or 128). D_lanes, when given, receives the raw contents of all 128 TMEM lanes.
template <int NB, bool BF16, int MG>
__global__ void __launch_bounds__(256) k_tc_selftest(const uint16_t* __restrict__ A, const uint16_t* __restrict__ Bm,
                                                     float* __restrict__ D, float* __restrict__ D_lanes,
                                                     DevStatus* status) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* A_s = base;
  uint8_t* B_s = base + kG * kKPix * 2;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(B_s + NB * kKPix * 2);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
  for (int e = threadIdx.x; e < MG * kKPix; e += blockDim.x) {
    const int m = e / kKPix, k = e % kKPix;
    *reinterpret_cast<uint16_t*>(A_s + kmajor_sw128(m, k, MG)) = A[e];
  }
  for (int e = threadIdx.x; e < NB * kKPix; e += blockDim.x) {
    const int nn = e / kKPix, k = e % kKPix;
    *reinterpret_cast<uint16_t*>(B_s + kmajor_sw128(nn, k, NB)) = Bm[e];
  }
  if (threadIdx.x == 0) mbar_init(mbar, 1);
  if (threadIdx.x < 32) {
    tmem_alloc(tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (threadIdx.x == 0) issue_batch<NB, MG>(smem_u32(A_s), smem_u32(B_s), tmem, idesc_f16(MG, NB, BF16), mbar);
  const bool ok = __all_sync(0xFFFFFFFFu, mbar_wait_bounded(mbar, 0));  // warp-uniform for tcgen05.ld
  if (!ok && (threadIdx.x & 31) == 0) atomicOr(&status->flags, kFlagTimeout);
  tc_fence_after();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < 4 && ok) {
    const int L = warp * 32 + lane;  // the TMEM lane this thread reads
    const int row = tmem_row_of_lane<MG>(warp, lane);
#pragma unroll
    for (int c0 = 0; c0 < NB; c0 += 16) {
      uint32_t r[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
      tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        if (row >= 0) D[row * NB + c0 + q] = __uint_as_float(r[q]);
        if (D_lanes) D_lanes[L * NB + c0 + q] = __uint_as_float(r[q]);
      }
    }
  }
  if (!ok) mbar_wait_bounded(mbar, 0);
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ---- the accumulate walk with the tensor-core contraction --------------------------------------
// MG: Gaussians per batch, the MMA M (128, or 64 for up to 32 channels: half the weight operand, so
// that more CTAs fit on an SM). TMEM columns: the accumulator width rounded up to a power of two.
// Columns of B and of the accumulator: the KT target channels, then rows of ones that yield V (16
// for M = 128, whose N must be a multiple of 16; 8 for M = 64, which allows multiples of 8).
template <int KT, int MG>
__host__ __device__ constexpr int tc_cols() {
  return KT + (MG == 64 ? 8 : 16);
}

template <int NB>
__host__ __device__ constexpr uint32_t tmem_cols() {
  return NB <= 32 ? 32u : (NB <= 64 ? 64u : 128u);
}

template <int KT, int MG>
__host__ __device__ constexpr int tc_ctas_per_sm() {
  return MG == 64 ? (KT <= 16 ? 5 : (KT <= 32 ? 4 : 3)) : 2;
}

template <int KT, bool BF16_TARGETS, int MG>
__global__ void __launch_bounds__(256, tc_ctas_per_sm<KT, MG>()) k_blend_accumulate_tc(
    const uint32_t* __restrict__ tile_off, const uint64_t* __restrict__ entries, uint32_t capacity,
    const ProjRec* __restrict__ rec, int64_t n, int width, int height, int tiles_x, int tiles,
    const uint16_t* __restrict__ targets, int K, int cam0, float* __restrict__ acc, int RS,
    int64_t acc_cam_stride, DevStatus* status, uint64_t wait_limit_ns, bool issue_mma) {
  static_assert(MG == 64, "staging and epilogue map Gaussian g to TMEM lane g % 16 of quarter g / 16 (M = 64)");
  constexpr int NB = tc_cols<KT, MG>();  // target channels + rows of ones (V)
  constexpr bool kB16 = KT == 16;        // B in the 11 KB region (b16_offset)
  extern __shared__ uint8_t smem_raw[];
  // The barrier and flags (48 bytes) sit in front of the 1024-byte aligned operands, inside the
  // 1 KB the layout allows for alignment: from a base that is 128-byte aligned the operands then
  // start at most 1024 bytes in. A base that is not is reported (kFlagLayout) before any work.
  const uint32_t raw = smem_u32(smem_raw);
  if (raw & 127u) {
    if (threadIdx.x == 0) atomicOr(&status->flags, kFlagLayout);
    return;
  }
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
  uint32_t* s_timeout = tmem_slot + 1;  // set by a thread whose wait gave up
  uint32_t* s_tmax = s_timeout + 1;     // [8]
  uint8_t* base = smem_raw + (((raw + 48u + 1023u) & ~1023u) - raw);
  uint8_t* A_s = base;                                 // MG x 256 (32 KB)
  uint8_t* B_s = base + MG * kKPix * 2;                // NB x 256, or the 11 KB region
  // The batch's geometry is read only by the pixel walk, which ends at the first barrier of the
  // batch: the next batch is staged into the same buffer while the MMAs run.
  float4* s_geo = reinterpret_cast<float4*>(kB16 ? B_s + kB16Geo : B_s + NB * kKPix * 2);  // [MG]
  float4* s_aux = kB16 ? reinterpret_cast<float4*>(B_s + kB16Aux) : s_geo + MG;             // [MG]

  const TileCtx c = tile_ctx(tile_off, capacity, tiles, tiles_x, width, height);
  if (c.len == 0) return;  // uniform: nothing binned to this tile
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tx0 = (c.t % tiles_x) * kTile, ty0 = (c.t / tiles_x) * kTile;
  const int p = (c.py - ty0) * kTile + (c.px - tx0);  // this thread's pixel index in the tile (MMA k)

  // B: the tile's targets, transposed to [channel][pixel] and scaled by 2^s (the tile's largest
  // magnitude in [2^14, 2^15)), then the rows of ones
  float t_scale_inv;
  {
    const uint16_t* src = targets + ((((int64_t)(cam0 + c.j) * height + c.py) * width + c.px) * K);
    // this pixel's channels, loaded 16 bytes at a time when the row allows it
    uint16_t tv[KT];
    if (c.inside && K == KT && (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
#pragma unroll
      for (int q = 0; q < KT / 8; ++q) {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(src) + q);
        const uint32_t wd[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          tv[8 * q + 2 * h] = (uint16_t)(wd[h] & 0xFFFFu);
          tv[8 * q + 2 * h + 1] = (uint16_t)(wd[h] >> 16);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < KT; ++k) tv[k] = (c.inside && k < K) ? src[k] : (uint16_t)0;
    }
    float tmax = 0.0f;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      const float x = target_value(tv[k], BF16_TARGETS);
      tmax = fmaxf(tmax, fabsf(x));
      bad |= !isfinite(x);
    }
    if (bad) atomicOr(&status->flags, kFlagNonfinite);
    // non-negative floats order like their bit patterns
    uint32_t m = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(tmax));
    if (lane == 0) s_tmax[warp] = m;
    __syncthreads();
    m = s_tmax[0];
#pragma unroll
    for (int w2 = 1; w2 < 8; ++w2) m = max(m, s_tmax[w2]);
    const float gmax = __uint_as_float(m);
    int e = 0;
    if (gmax > 0.0f && isfinite(gmax)) frexpf(gmax, &e);  // gmax in [2^(e-1), 2^e)
    const int sexp = gmax > 0.0f ? 15 - e : 0;           // gmax * 2^sexp in [2^14, 2^15)
    t_scale_inv = ldexpf(1.0f, -(sexp + kWScaleExp));
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      const float v = ldexpf(target_value(tv[k], BF16_TARGETS), sexp);
      *reinterpret_cast<uint16_t*>(B_s + (kB16 ? b16_offset(k, p) : kmajor_sw128(k, p, NB))) = half_bits(v);
    }
    if constexpr (kB16) {
      if (threadIdx.x < 64)
        reinterpret_cast<uint4*>(B_s + kB16Ones)[threadIdx.x] = make_uint4(0x3C003C00u, 0x3C003C00u, 0x3C003C00u, 0x3C003C00u);
    } else {
#pragma unroll
      for (int k = KT; k < NB; ++k) *reinterpret_cast<uint16_t*>(B_s + kmajor_sw128(k, p, NB)) = (uint16_t)0x3C00u;
    }
  }
  const float v_scale_inv = ldexpf(1.0f, -kWScaleExp);
  const ProjRec* rec_cam = rec + (int64_t)c.j * n;
  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    *s_timeout = 0u;
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, tmem_cols<NB>());
    tmem_relinquish();
  }
  // the first batch's staging, and W cleared
  constexpr int kCh = KT / 16;          // 16-column chunks of S in the epilogue
  constexpr int kHalf = (kCh + 1) / 2;  // chunks of the warps 0-3
  const int g_own = tmem_row_of_lane<MG>(warp & 3, lane);  // the batch row this thread stages and adds
  const bool stager = warp < 4, need_id = warp < 4 || kCh > kHalf;
  const unsigned long long* list = reinterpret_cast<const unsigned long long*>(entries);
  uint32_t my_id = stage_tc(list, c.b, (int)min((uint32_t)MG, c.len), rec_cam, n, c.ox, c.oy, s_geo, s_aux, g_own,
                            stager, need_id);
  for (int i = threadIdx.x; i < MG * kKPix * 2 / 16; i += 256) reinterpret_cast<uint4*>(A_s)[i] = make_uint4(0, 0, 0, 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t a_addr = smem_u32(A_s), b_addr = smem_u32(B_s);
  constexpr uint32_t kIdesc = idesc_f16(MG, NB, false);
  float* acc_cam = acc + (int64_t)c.j * acc_cam_stride;
  float T = (float)(1 << kWScaleExp);  // the transmittance times 2^14 (blend_take)
  bool done = !c.inside;
  // kmajor_sw128(g, p, MG) split into this pixel's part and the Gaussian's: the row's 128 bytes at
  // g * 128 (8-row atoms of 1024 bytes), the 16-byte chunk (p % 64) / 8 XOR-ed with g % 8
  uint8_t* const a_pix = A_s + (p >> 6) * (MG * 128) + ((p & 7) << 1);
  const int a_chunk = ((p & 63) >> 3) << 4;
  uint32_t npairs = 0, phase = 0;
  // Two CTA barriers per batch: one before the MMA issue (W written), one at the end (the next
  // batch's staging loaded, W cleared, the done count and the timeout flag published).
  for (uint32_t start = 0, buf = 0; start < c.len; start += MG, buf ^= 1u) {
    const int nb = (int)min((uint32_t)MG, c.len - start);
    if (!__all_sync(0xFFFFFFFFu, done)) {
#pragma unroll
      for (int q = 0; q < MG / 32; ++q) {
        uint32_t bits = warp_hit_bits_packed(s_geo, s_aux, q * 32, nb, c);
        while (bits && !done) {  // two hits a step: both alphas first (independent of T)
          const int g1 = q * 32 + __ffs(bits) - 1;
          bits &= bits - 1;
          const bool has2 = bits != 0;  // warp-uniform
          const int g2 = has2 ? q * 32 + __ffs(bits) - 1 : g1;
          bits &= bits - 1;
          const float4 aux1 = s_aux[g1], aux2 = s_aux[g2];
          const StepAlpha a1 = blend_alpha_noreject(s_geo[g1], aux1, c.pxf, c.pyf);
          StepAlpha a2 = blend_alpha_noreject(s_geo[g2], aux2, c.pxf, c.pyf);
          a2.ok = a2.ok && has2;
          // T carries the factor 2^14 of W, so the weights come out scaled
          const float w1 = blend_take<false, kWScaleExp>(a1, T, done, npairs);
          const float w2 = blend_take<true, kWScaleExp>(a2, T, done, npairs);
          // the staged row offset XOR this pixel's chunk: kmajor_sw128(g, p, MG) - (a_pix - A_s)
          *reinterpret_cast<uint16_t*>(a_pix + (__float_as_uint(aux1.z) ^ a_chunk)) = half_bits(w1);
          if (has2) *reinterpret_cast<uint16_t*>(a_pix + (__float_as_uint(aux2.z) ^ a_chunk)) = half_bits(w2);
        }
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && issue_mma) {
      if constexpr (kB16) issue_batch_b16<MG>(a_addr, b_addr, tmem, kIdesc, mbar);
      else issue_batch<NB, MG>(a_addr, b_addr, tmem, kIdesc, mbar);
    }
    // while the MMAs run: stage the next batch (the pixel walk of this one has ended; each
    // thread keeps this batch's index for the epilogue)
    const uint32_t next = start + MG;
    uint32_t next_id = 0;
    if (next < c.len)
      next_id = stage_tc(list, c.b + next, (int)min((uint32_t)MG, c.len - next), rec_cam, n, c.ox, c.oy, s_geo, s_aux,
                         g_own, stager, need_id);
    // warp-uniform: the epilogue's tcgen05.ld needs whole warps
    const bool ok = __all_sync(0xFFFFFFFFu, mbar_wait_bounded(mbar, phase, wait_limit_ns));
    phase ^= 1u;
    tc_fence_after();
    if (ok) {
      // warps w and w+4 share TMEM lanes 32(w%4)..+31 (one Gaussian per thread) and split its 16-column
      // chunks; with MG = 64 only the first 16 lanes of each quarter hold a Gaussian (tmem_row_of_lane).
      // The accumulator streams through registers a chunk at a time: chunk c adds the float4 groups
      // 4c..4c+3 of the row (V, S_0, S_1, ..) and carries its last column into group 4c+4. Every
      // tcgen05.ld is warp-uniform; only the atomics depend on the thread's Gaussian.
      const int quarter = warp & 3, part = warp >> 2;
      const int g = g_own;
      const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
      if (part == 0 || kCh > kHalf) {        // warp-uniform
        uint32_t vr[16], r[16];
        tmem_ld16(trow + (uint32_t)KT, vr);  // the ones block: every column holds V
        if (part == 1) tmem_ld16(trow + (uint32_t)(16 * (kHalf - 1)), r);  // the column before this part
        tmem_wait_ld();
        const float V = __uint_as_float(vr[0]) * v_scale_inv;
        float carry = part == 0 ? V : __uint_as_float(r[15]) * t_scale_inv;
        const bool add = g >= 0 && g < nb && V > 0.0f;
        float* dst = acc_cam + (int64_t)(add ? my_id : 0u) * RS;
        const int c_begin = part == 0 ? 0 : kHalf, c_end = part == 0 ? kHalf : kCh;
#pragma unroll
        for (int c = 0; c < kCh; ++c) {
          if (c < c_begin || c >= c_end) continue;  // warp-uniform
          tmem_ld16(trow + (uint32_t)(16 * c), r);
          tmem_wait_ld();
          float sv[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) sv[q] = __uint_as_float(r[q]) * t_scale_inv;
          if (add) {
            float* d = dst + 16 * c;
            if (16 * c < RS) atomicAdd(reinterpret_cast<float4*>(d), make_float4(carry, sv[0], sv[1], sv[2]));
            if (16 * c + 4 < RS) atomicAdd(reinterpret_cast<float4*>(d + 4), make_float4(sv[3], sv[4], sv[5], sv[6]));
            if (16 * c + 8 < RS) atomicAdd(reinterpret_cast<float4*>(d + 8), make_float4(sv[7], sv[8], sv[9], sv[10]));
            if (16 * c + 12 < RS)
              atomicAdd(reinterpret_cast<float4*>(d + 12), make_float4(sv[11], sv[12], sv[13], sv[14]));
          }
          carry = sv[15];
        }
        // the last group (S_{KT-1}, 0, 0, 0), by the warps that folded the last chunk
        if (add && part == (kCh > kHalf ? 1 : 0) && 16 * kCh < RS)
          atomicAdd(reinterpret_cast<float4*>(dst + 16 * kCh), make_float4(carry, 0.0f, 0.0f, 0.0f));
      }
    }
    my_id = next_id;
    if (!ok) {
      *s_timeout = 1u;
    } else if (next < c.len) {
      // this batch's MMAs have completed: clear W for the next batch (16-byte stores)
      for (int i = threadIdx.x; i < MG * kKPix * 2 / 16; i += 256) reinterpret_cast<uint4*>(A_s)[i] = make_uint4(0, 0, 0, 0);
    }
    tc_fence_before();
    const int n_done = __syncthreads_count(done);
    if (*s_timeout) {
      if (threadIdx.x == 0) atomicOr(&status->flags, kFlagTimeout);
      mbar_wait_bounded(mbar, phase ^ 1u, wait_limit_ns);  // give the outstanding MMAs a last chance to finish
      break;
    }
    if (n_done == (int)blockDim.x) break;
  }
  const uint32_t warp_sum = __reduce_add_sync(0xFFFFFFFFu, npairs);
  if (lane == 0 && warp_sum) atomicAdd((unsigned long long*)&status->contrib_pairs, (unsigned long long)warp_sum);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, tmem_cols<NB>());
  }
}

template <int NB>
constexpr size_t selftest_smem() {
  return 1024 + (size_t)kG * kKPix * 2 + (size_t)NB * kKPix * 2 + 16;
}
// the barrier and flags with the alignment slack (1 KB), W, and B (with the staged geometry in its
// holes at 16 channels, after it otherwise)
template <int KT, int MG>
constexpr size_t tc_smem() {
  return 1024 + (size_t)MG * kKPix * 2 +
         (KT == 16 ? (size_t)kB16Bytes : (size_t)tc_cols<KT, MG>() * kKPix * 2 + (size_t)MG * 32);
}
// CTAs per SM that the shared memory admits: each CTA's share rounded up to 1 KB, plus 1 KB the
// system reserves per CTA, out of the SM's 228 KB
template <int KT, int MG>
constexpr int tc_smem_ctas() {
  return (int)((228 * 1024) / ((tc_smem<KT, MG>() + 1023) / 1024 * 1024 + 1024));
}
static_assert(tc_smem_ctas<16, 64>() >= tc_ctas_per_sm<16, 64>(), "shared memory of the 16-channel walk");
static_assert(tc_smem_ctas<32, 64>() >= tc_ctas_per_sm<32, 64>(), "shared memory of the 32-channel walk");
static_assert(tc_smem_ctas<64, 64>() >= tc_ctas_per_sm<64, 64>(), "shared memory of the 64-channel walk");

// Diagnostic settings of this host thread (icgs_debug_tc_wait): the walk's wait limit and whether
// it issues its MMAs.
thread_local uint64_t g_wait_limit_ns = kWaitLimitNs;
thread_local bool g_issue_mma = true;

template <int KT, bool BF16_TARGETS>
void accumulate_tc(const Problem& p, int cb, int cam0, const void* targets, const Workspace& ws, cudaStream_t s) {
  constexpr int MG = 64;
  const size_t smem = tc_smem<KT, MG>();
  cudaFuncSetAttribute(k_blend_accumulate_tc<KT, BF16_TARGETS, MG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  cudaFuncSetAttribute(k_blend_accumulate_tc<KT, BF16_TARGETS, MG>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
  const int64_t stride = p.L == 0 ? 0 : p.n * (int64_t)p.acc_stride;
  k_blend_accumulate_tc<KT, BF16_TARGETS, MG><<<cb * p.tiles, 256, smem, s>>>(
      ws.tile_off, ws.entries, p.capacity, ws.rec, p.n, p.width, p.height, p.tiles_x, p.tiles,
      static_cast<const uint16_t*>(targets), p.K, cam0, ws.acc, p.acc_stride, stride, ws.status, g_wait_limit_ns,
      g_issue_mma);
  note_launches(1);
}

template <bool BF16_TARGETS>
void accumulate_tc_dispatch(const Problem& p, int cb, int cam0, const void* targets, const Workspace& ws,
                            cudaStream_t s) {
  if (p.K <= 16) accumulate_tc<16, BF16_TARGETS>(p, cb, cam0, targets, ws, s);
  else if (p.K <= 32) accumulate_tc<32, BF16_TARGETS>(p, cb, cam0, targets, ws, s);
  else accumulate_tc<64, BF16_TARGETS>(p, cb, cam0, targets, ws, s);
}

}  // namespace

void set_tc_wait_diagnostic(int64_t limit_ns, bool issue_mma) {
  g_wait_limit_ns = limit_ns > 0 ? (uint64_t)limit_ns : kWaitLimitNs;
  g_issue_mma = issue_mma;
}

bool tc_accumulate_applies(const Problem& p, int dtype) {
  return p.precision == 1 && (dtype == 1 || dtype == 2) && p.K >= 16 && p.K <= 64;
}

void launch_blend_accumulate_tc(const Problem& p, int cb, int cam0, const void* targets, int dtype,
                                const Workspace& ws, cudaStream_t s) {
  if (dtype == 1) accumulate_tc_dispatch<true>(p, cb, cam0, targets, ws, s);
  else accumulate_tc_dispatch<false>(p, cb, cam0, targets, ws, s);
}

cudaError_t launch_tc_selftest(const uint16_t* A, int M, const uint16_t* B, int N, bool bf16, float* D, float* D_lanes,
                               DevStatus* status, cudaStream_t s) {
#define ICGS_ST(NB, BF, MG)                                                                                    \
  do {                                                                                                         \
    cudaFuncSetAttribute(k_tc_selftest<NB, BF, MG>, cudaFuncAttributeMaxDynamicSharedMemorySize,             \
                         (int)selftest_smem<NB>());                                                           \
    k_tc_selftest<NB, BF, MG><<<1, 256, selftest_smem<NB>(), s>>>(A, B, D, D_lanes, status);                   \
  } while (0)
#define ICGS_ST_M(NB, BF)                \
  do {                                   \
    if (M == 64) ICGS_ST(NB, BF, 64);    \
    else ICGS_ST(NB, BF, 128);           \
  } while (0)
  if (M != 64 && M != 128) return cudaErrorInvalidValue;
  if (N == 32 && bf16) ICGS_ST_M(32, true);
  else if (N == 32) ICGS_ST_M(32, false);
  else if (N == 80 && bf16) ICGS_ST_M(80, true);
  else if (N == 80) ICGS_ST_M(80, false);
  else return cudaErrorInvalidValue;
#undef ICGS_ST_M
#undef ICGS_ST
  return cudaGetLastError();
}

}  // namespace icgs
