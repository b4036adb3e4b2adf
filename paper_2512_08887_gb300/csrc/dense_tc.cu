// Dense stage 2 on the tensor cores (Sec. III-B "precompute" variant, Table I): for every beam b
//   bhat_b[:, blk] = G_b w_b[blk],   G_b = F_u A_b^{-1}  (N x L complex, built in FP64 at plan time).
//
// Per beam the blocks form the right-hand sides of a complex GEMM (N x L) . (L x nblk). It runs as
// four real products on split real/imaginary planes, so neither operand is duplicated:
//   C_re = G_re W_re - G_im W_im,   C_im = G_re W_im + G_im W_re,
// the subtraction done by the negate-B bit of the MMA instruction descriptor. Precision variants:
//   BF16X3 : G = G_hi + G_lo, W = W_hi + W_lo in BF16; hi*hi + hi*lo + lo*hi per product (kind::f16)
//   TF32   : G, W rounded to TF32, one product (kind::tf32)
//   TF32X3 : G = G_hi + G_lo, W = W_hi + W_lo with TF32 hi parts and FP32 residuals (kind::tf32),
//            hi*hi + hi*lo + lo*hi: FP32-class accuracy
// always with FP32 accumulation in tensor memory.
//
// Long sums in TF32 lose accuracy as K = L grows, so k_dense_tc spreads the K chunks over KACC
// partial accumulators in tensor memory (chunk c adds into accumulator c % KACC, up to 4 of them
// within the 512 columns) and the epilogue adds the partials in FP32.
//
// BF16X3 and TF32 (k_dense_tc: one CTA = one beam x 128 output samples x up to NB blocks, 128
// threads) read operands that separate kernels have already split into planes:
//   thread 0  : TMA producer (cp.async.bulk.tensor, 128-byte swizzle, one mbarrier per stage)
//   thread 32 : MMA issuer (tcgen05.mma, cta_group::1, M = 128, N = NB, K = 32 bytes per step)
//   warp 1    : tensor-memory allocation / release (2 x NB columns per accumulator, KACC of them)
//   warps 0-3 : epilogue (tcgen05.ld 32x32b, rows = samples, coalesced complex64 stores)
// TF32X3 (k_dense_tc_fused, 384 or 256 threads) reads plain FP32 planes of G and the stage-1 output w as
// it is (interleaved complex64) and splits both on chip, so no split pass goes through HBM: the
// split G goes to tensor memory (the MMA's A operand), the split w to shared memory with the real
// and imaginary parts stacked along N, so each MMA is 128 x 2NB; see the kernel's own comment.
// Every mbarrier wait is bounded by %globaltimer; on timeout the kernel records FBST_ERR_TIMEOUT
// in the plan's status word, waits (bounded) for its copies in flight, frees its tensor memory
// and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <climits>
#include <mutex>

#include "common.cuh"
#include "launch_util.cuh"

namespace fbst {

enum tc_variant { TC_BF16X3 = 0, TC_TF32 = 1, TC_TF32X3 = 2, TC_F16X3 = 3 };

template <int V> struct tc_traits;
template <> struct tc_traits<TC_BF16X3> {
  static constexpr int ESZ = 2, NPL = 4, TERMS = 3, MAX_NB = 64, STAGES = 2;
  static constexpr uint32_t FMT = 1;  // BF16
};
template <> struct tc_traits<TC_TF32> {
  static constexpr int ESZ = 4, NPL = 2, TERMS = 1, MAX_NB = 128, STAGES = 3;
  static constexpr uint32_t FMT = 2;  // TF32
};
template <> struct tc_traits<TC_TF32X3> {
  static constexpr int ESZ = 4, NPL = 4, TERMS = 3, MAX_NB = 64, STAGES = 2;
  static constexpr uint32_t FMT = 2;  // TF32
};

static int variant_of(int stage2) {
  switch (stage2) {
    case FBST_STAGE2_DENSE_BF16X3: return TC_BF16X3;
    case FBST_STAGE2_DENSE_TF32: return TC_TF32;
    case FBST_STAGE2_DENSE_TF32X3: return TC_TF32X3;
    case FBST_STAGE2_DENSE_F16X3: return TC_F16X3;
    default: return -1;
  }
}

constexpr int kRowBytes = 128;    // one K-chunk row (the 128-byte swizzle span)
constexpr int kTileM = 128;       // output samples per CTA (MMA M)
constexpr int kWParts = 16;       // CTAs per block of w that find its largest magnitude (FP16 split)
constexpr uint64_t kWaitNs = 1000000000ull;   // default limit of a pipeline wait (1 s; per plan)
constexpr uint64_t kDrainNs = 2000000000ull;  // limit of the waits that drain copies / MMAs in flight

// ---------------------------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity; false if it did not complete within limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() - t0 > limit_ns) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor, K-major operand in the 128-byte swizzle layout written by TMA:
// rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor: FP32 accumulator, A/B format, optional negation of B, both K-major,
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, int M, int N, bool neg_b) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((neg_b ? 1u : 0u) << 14) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <int V>
__device__ __forceinline__ void mma_issue(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  if constexpr (V == TC_BF16X3) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The same load without the wait: several loads may be in flight before one tmem_wait_ld().
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t h2_bits(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }

__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// ---------------------------------------------------------------------------------------------
// Operand preparation
// ---------------------------------------------------------------------------------------------
// Split one FP32 value into the variant's planes (hi, lo) or (rounded).
template <int V>
__device__ __forceinline__ void split_store(void* base, size_t plane_stride, size_t idx, int comp, float x) {
  if constexpr (V == TC_BF16X3) {
    __nv_bfloat16* p = static_cast<__nv_bfloat16*>(base);
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
    p[(size_t)(2 * comp) * plane_stride + idx] = hi;
    p[(size_t)(2 * comp + 1) * plane_stride + idx] = lo;
  } else if constexpr (V == TC_TF32) {
    static_cast<float*>(base)[(size_t)comp * plane_stride + idx] = round_tf32(x);
  } else {
    const float hi = round_tf32(x);
    static_cast<float*>(base)[(size_t)(2 * comp) * plane_stride + idx] = hi;
    static_cast<float*>(base)[(size_t)(2 * comp + 1) * plane_stride + idx] = x - hi;
  }
}

// G [B][N][L] complex64 -> planes [B][NPL][N][L].
template <int V>
__global__ void k_tc_split_G(const float2* __restrict__ G, void* __restrict__ out, int B, int N, int L) {
  constexpr int NPL = tc_traits<V>::NPL;
  const size_t per_beam = (size_t)N * L;
  const size_t total = (size_t)B * per_beam;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / per_beam, r = i % per_beam;
    const float2 g = G[i];
    char* beam = static_cast<char*>(out) + b * NPL * per_beam * tc_traits<V>::ESZ;
    split_store<V>(beam, per_beam, r, 0, g.x);
    split_store<V>(beam, per_beam, r, 1, g.y);
  }
}

// w [nblk][B][L] complex64 -> planes [B][NPL][NBW][L]; rows nblk..nrows-1 are zero.
template <int V>
__global__ void k_tc_prep_w(const float2* __restrict__ w, void* __restrict__ out, int B, int L, int nblk, int nrows,
                            int NBW) {
  constexpr int NPL = tc_traits<V>::NPL;
  const int b = blockIdx.y;
  const size_t plane = (size_t)NBW * L;
  char* beam = static_cast<char*>(out) + (size_t)b * NPL * plane * tc_traits<V>::ESZ;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nrows * L; i += gridDim.x * blockDim.x) {
    const int blk = i / L, l = i % L;
    const float2 v = blk < nblk ? w[((size_t)blk * B + b) * L + l] : make_float2(0.f, 0.f);
    split_store<V>(beam, plane, (size_t)blk * L + l, 0, v.x);
    split_store<V>(beam, plane, (size_t)blk * L + l, 1, v.y);
  }
}

// ---------------------------------------------------------------------------------------------
// The GEMM kernel
// ---------------------------------------------------------------------------------------------
template <int V, int NB>
struct tc_smem {
  static constexpr int NPL = tc_traits<V>::NPL;
  static constexpr int STAGES = tc_traits<V>::STAGES;
  static constexpr int A_TILE = kTileM * kRowBytes;   // one plane
  static constexpr int B_TILE = NB * kRowBytes;
  static constexpr int STAGE_BYTES = NPL * (A_TILE + B_TILE);
  static constexpr int BYTES = STAGES * STAGE_BYTES + 1024 /* alignment slack */ + 256 /* barriers */;
};

template <int V, int NB>
__global__ void __launch_bounds__(128, 1)
k_dense_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
           float2* __restrict__ bhat, int B, int N, int L, int nblk, int* status, uint64_t wait_ns) {
  using TR = tc_traits<V>;
  using SM = tc_smem<V, NB>;
  constexpr int NPL = TR::NPL, STAGES = TR::STAGES;
  constexpr int KELEM = kRowBytes / TR::ESZ;      // elements per K-chunk row
  constexpr int KSTEPS = kRowBytes / 32;          // MMAs of 32 bytes of K per chunk
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * SM::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTileM, b = blockIdx.y, blk0 = blockIdx.z * NB;
  const int nchunks = (L + KELEM - 1) / KELEM;
  // KACC partial accumulators (K-chunk c goes to accumulator c % KACC), summed in FP32 in the
  // epilogue: the tensor pipe's accumulation error grows with the number of terms it sums, so
  // shorter partial sums keep the split-precision variants near FP32 accuracy.
  constexpr int KACC = 2 * NB * 4 <= 512 ? 4 : (2 * NB * 2 <= 512 ? 2 : 1);
  constexpr uint32_t COLS = 2 * NB * KACC;
  constexpr uint32_t TMEM_COLS = COLS <= 32 ? 32 : (COLS <= 64 ? 64 : (COLS <= 128 ? 128 : (COLS <= 256 ? 256 : 512)));

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (threadIdx.x == 0) {
    // ---------------- TMA producer ----------------
    int issued = 0;
    for (int c = 0; c < nchunks; ++c) {
      const int s = c % STAGES;
      if (c >= STAGES && !mbar_wait(&empty[s], ((c / STAGES) - 1) & 1, wait_ns)) {
        atomicExch(status, (int)FBST_ERR_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      uint8_t* st = smem + s * SM::STAGE_BYTES;
      mbar_expect_tx(&full[s], SM::STAGE_BYTES);
      for (int pl = 0; pl < NPL; ++pl) {
        tma_load_3d(st + pl * SM::A_TILE, &mapA, &full[s], c * KELEM, m0, b * NPL + pl);
        tma_load_3d(st + NPL * SM::A_TILE + pl * SM::B_TILE, &mapB, &full[s], c * KELEM, blk0, b * NPL + pl);
      }
      issued = c + 1;
    }
    // Copies still in flight must land before the CTA can leave (on the normal path these phases
    // have completed already and the waits return at once).
    for (int c = (issued > STAGES ? issued - STAGES : 0); c < issued; ++c)
      (void)mbar_wait(&full[c % STAGES], (c / STAGES) & 1, kDrainNs);
  } else if (threadIdx.x == 32) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t ID_POS = make_idesc(TR::FMT, kTileM, NB, false);
    constexpr uint32_t ID_NEG = make_idesc(TR::FMT, kTileM, NB, true);
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int s = c % STAGES;
      if (!mbar_wait(&full[s], (c / STAGES) & 1, wait_ns)) {
        atomicExch(status, (int)FBST_ERR_TIMEOUT);
        *abort_flag = 1;
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = smem_u32(smem + s * SM::STAGE_BYTES);
      const uint32_t d_re = tmem + (uint32_t)((c % KACC) * 2 * NB), d_im = d_re + NB;
      // Planes: TERMS == 1 -> {re, im}; TERMS == 3 -> {re_hi, re_lo, im_hi, im_lo}.
      constexpr int RE_HI = 0, RE_LO = (TR::TERMS == 3 ? 1 : 0), IM_HI = (TR::TERMS == 3 ? 2 : 1),
                    IM_LO = (TR::TERMS == 3 ? 3 : 1);
#pragma unroll
      for (int k = 0; k < KSTEPS; ++k) {
        auto da = [&](int pl) { return smem_desc_sw128(st + pl * SM::A_TILE + k * 32); };
        auto db = [&](int pl) { return smem_desc_sw128(st + NPL * SM::A_TILE + pl * SM::B_TILE + k * 32); };
        const uint32_t acc0 = (c >= KACC || k > 0) ? 1u : 0u;
        // C_re = G_re W_re - G_im W_im ; C_im = G_re W_im + G_im W_re
        mma_issue<V>(d_re, da(RE_HI), db(RE_HI), ID_POS, acc0);
        mma_issue<V>(d_re, da(IM_HI), db(IM_HI), ID_NEG, 1u);
        mma_issue<V>(d_im, da(RE_HI), db(IM_HI), ID_POS, acc0);
        mma_issue<V>(d_im, da(IM_HI), db(RE_HI), ID_POS, 1u);
        if constexpr (TR::TERMS == 3) {
          mma_issue<V>(d_re, da(RE_HI), db(RE_LO), ID_POS, 1u);
          mma_issue<V>(d_re, da(RE_LO), db(RE_HI), ID_POS, 1u);
          mma_issue<V>(d_re, da(IM_HI), db(IM_LO), ID_NEG, 1u);
          mma_issue<V>(d_re, da(IM_LO), db(IM_HI), ID_NEG, 1u);
          mma_issue<V>(d_im, da(RE_HI), db(IM_LO), ID_POS, 1u);
          mma_issue<V>(d_im, da(RE_LO), db(IM_HI), ID_POS, 1u);
          mma_issue<V>(d_im, da(IM_HI), db(RE_LO), ID_POS, 1u);
          mma_issue<V>(d_im, da(IM_LO), db(RE_HI), ID_POS, 1u);
        }
      }
      mma_commit(&empty[s]);  // this stage's smem may be refilled once these MMAs have read it
    }
    mma_commit(done);  // all issued MMAs complete -> accumulators final
  }
  __syncwarp();

  // ---------------- Epilogue: all four warps ----------------
  const bool have = mbar_wait(done, 0, wait_ns);
  if (!have) {
    if (lane == 0) atomicExch(status, (int)FBST_ERR_TIMEOUT);
    *abort_flag = 1;
    // The MMAs already issued must finish before tensor memory is released.
    (void)mbar_wait(done, 0, kDrainNs);
  } else if (!*abort_flag) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int n = m0 + warp * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    const int nacc = nchunks < KACC ? nchunks : KACC;
#pragma unroll 1
    for (int j0 = 0; j0 < NB; j0 += 16) {
      float re[16], im[16];
      tmem_ld16(lane_base + j0, re);
      tmem_ld16(lane_base + NB + j0, im);
      for (int q = 1; q < nacc; ++q) {
        float re2[16], im2[16];
        tmem_ld16(lane_base + q * 2 * NB + j0, re2);
        tmem_ld16(lane_base + q * 2 * NB + NB + j0, im2);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          re[jj] += re2[jj];
          im[jj] += im2[jj];
        }
      }
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int blk = blk0 + j0 + jj;
        if (blk < nblk && n < N) bhat[((size_t)blk * B + b) * N + n] = make_float2(re[jj], im[jj]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ---------------------------------------------------------------------------------------------
// Fused TF32x3 kernel. The plan keeps G_b as plain FP32 real/imaginary planes; the kernel reads
// them and the interleaved complex64 w tiles of stage 1 straight by TMA and splits both on chip:
//   * G (the MMA's A operand) goes to tensor memory: for every K step of 8 values a converter
//     thread owns one row, rounds it to TF32 (hi) and keeps the FP32 residual (lo), and stores
//     [hi_re | hi_im | lo_re | lo_im] (4 x 8 columns) into a ring of 4 tensor-memory slots with
//     tcgen05.st. The MMAs take A from tensor memory, so shared memory only feeds B.
//   * w (the B operand) is deinterleaved into two stacked planes per stage, hi and lo, each of
//     3*NB rows [-W_im | W_re | W_im] in the 128-byte swizzle layout. Rows NB..3NB are
//     [W_re | W_im] and rows 0..2NB are [-W_im | W_re], so one MMA of N = 2*NB gives
//     A_re [W_re | W_im] and another A_im [-W_im | W_re]; their sum is [C_re | C_im]. (Two MMAs of
//     N = NB with the negate-B bit instead need a smaller plane but run slower per MAC.)
// Per K step: 2 MMAs of hi*hi into accumulator H[chunk parity] and 4 of hi*lo / lo*hi into
// accumulator LO (terms 2^-11 smaller, so their rounding does not matter); the epilogue adds
// H0 + H1 + LO in FP32. Splitting the large hi*hi sum over two accumulators keeps the growth of
// the accumulation error with L in check.
// The converters copy a chunk's G rows to registers and release its raw TMA stage before they
// wait for tensor-memory slots, so the next TMA load is not held up by the MMAs.
// PERSIST: one CTA per SM walks tiles (beam x 128 samples x up to NB blocks) with stride
// gridDim.x; the TMA, conversion and tensor-memory rings run on across tiles, and the epilogue
// warps release the accumulators (tempty) as soon as they have read them, so the next tile's loads
// and conversions overlap the previous tile's MMAs and stores. Without PERSIST (256 threads, one
// tile per CTA, two CTAs per SM) warps 0-3 run the epilogue after the main loop.
//   thread 0   : TMA producer (raw stage ring, freed by the converters once read)
//   thread 32  : MMA issuer; warp 1 allocates and frees tensor memory
//   warps 4-7  : converters (thread = A row = tensor-memory lane)
//   warps 8-11 : epilogue (tcgen05.ld, FP32 sums, coalesced complex64 stores; warps 0-3 without
//                PERSIST)
//   warps 2-3  : idle until the epilogue
// ---------------------------------------------------------------------------------------------
template <int NB, bool F16>
struct fused_smem {
  // The FP16 planes are half the size, so a persistent CTA (NB >= 32) fits one more raw stage.
  static constexpr int RAW_STAGES = (F16 && NB >= 32) ? 3 : 2, PL_STAGES = 2;
  static constexpr int A_TILE = kTileM * kRowBytes;         // one FP32 plane of G: 128 rows x 32 K values
  static constexpr int W_BOX = NB * kRowBytes;              // raw w: NB rows x 16 complex values
  static constexpr int RAW_BYTES = 2 * A_TILE + 2 * W_BOX;  // TMA bytes of one stage (re, im, 2 w boxes)
  static constexpr int WROW = F16 ? 64 : kRowBytes;         // bytes of a 32-value K row of a w plane
  static constexpr int WPL = 3 * NB * WROW;                 // one stacked plane [-W_im | W_re | W_im]
  static constexpr int PL_OFF = RAW_STAGES * RAW_BYTES;     // W planes: PL_STAGES x {hi, lo}
  static constexpr int BAR_OFF = PL_OFF + PL_STAGES * 2 * WPL;
  static constexpr int BAR_BYTES = 512;                     // mbarriers, tensor-memory slot, abort flag
  static constexpr int BYTES = BAR_OFF + BAR_BYTES + 1024;  // + alignment slack
  static_assert(RAW_BYTES % 1024 == 0 && WPL % 1024 == 0, "1024-byte aligned swizzle atoms");
  static_assert(BYTES <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ float4 rna4(float4 x) {
  return make_float4(round_tf32(x.x), round_tf32(x.y), round_tf32(x.z), round_tf32(x.w));
}
__device__ __forceinline__ float4 sub4(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
__device__ __forceinline__ float4 neg4(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }

// TF32 MMA with A in tensor memory, B from a shared-memory descriptor.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(acc));
}

// FP16 MMA (K = 16) with A in tensor memory (two FP16 values per 32-bit column, the lower K index
// in the low half), B from a shared-memory descriptor.
__device__ __forceinline__ void mma_f16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                           uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(acc));
}

// Shared-memory matrix descriptor, K-major operand in the 64-byte swizzle layout: rows of 64 bytes,
// 8-row groups 512 bytes apart, 16-byte chunk c of row r stored at chunk c ^ ((r >> 1) & 3)
// (address bits 4-5 XOR bits 7-8), version 1, swizzle mode 4.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// 2^e as a float, for |e| <= 126 (exact).
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// The exponent e of the scale 2^e that maps a largest magnitude m into [2^14, 2^15) (frexp(m) =
// f 2^x with f in [0.5, 1) gives e = 15 - x), so that every scaled value is below 2^15 and fits
// FP16; 0 for m = 0 or a non-finite m.
__host__ __device__ __forceinline__ int scale_exp(float m) {
  if (!(m > 0.f) || !(m <= 3.4e38f)) return 0;
  int x;
  (void)frexpf(m, &x);
  const int e = 15 - x;
  return e < -120 ? -120 : (e > 120 ? 120 : e);
}

// The scale exponent of block blk from its largest |re|, |im| (float bits).
__device__ __forceinline__ int block_scale_exp(const unsigned* __restrict__ wmax, int blk) {
  return scale_exp(__uint_as_float(wmax[blk]));
}

// 16 consecutive 32-bit columns of this warp's 32 lanes (one value per thread and column).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

template <int NB, bool PERSIST, bool F16>
__global__ void __launch_bounds__(PERSIST ? 384 : 256, PERSIST ? 1 : 2)
k_dense_tc_fused(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapW,
                 float2* __restrict__ bhat, int B, int N, int L, int nblk, int b0, int nbeam, int w_beam_mul,
                 const int* __restrict__ gexp, const unsigned* __restrict__ wmax, int* status, uint64_t wait_ns) {
  using SM = fused_smem<NB, F16>;
  constexpr int RS = SM::RAW_STAGES, PS = SM::PL_STAGES;
  constexpr int KELEM = kRowBytes / 4;      // 32 FP32 values of K per chunk
  constexpr int KSTEPS = KELEM / (F16 ? 16 : 8);  // MMAs of K = 8 (TF32) or 16 (FP16) per chunk and term
  constexpr uint32_t RING = 0, H0 = 32 * KSTEPS, H1 = H0 + 2 * NB, LO = H1 + 2 * NB;
  constexpr uint32_t COLS = LO + 2 * NB;
  constexpr uint32_t TMEM_COLS = COLS <= 256 ? 256 : 512;
  static_assert(COLS <= 512, "tensor memory holds 512 columns");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + SM::BAR_OFF);
  uint64_t* rawfree = full + RS;
  uint64_t* wconv = rawfree + RS;
  uint64_t* wfree = wconv + PS;
  uint64_t* aready = wfree + PS;
  uint64_t* afree = aready + KSTEPS;
  uint64_t* tfull = afree + KSTEPS;  // a tile's accumulators are complete
  uint64_t* tempty = tfull + 1;      // the epilogue has read them
  uint64_t* mdone = tempty + 1;      // every MMA of this CTA has completed (before tensor memory is freed)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mdone + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = (L + KELEM - 1) / KELEM;
  const int mtiles = (N + kTileM - 1) / kTileM, ntiles = mtiles * nbeam * ((nblk + NB - 1) / NB);
  // Tile ti: row tile ti % mtiles, beam b0 + (ti / mtiles) % nbeam, block group ti / (mtiles nbeam)
  // (beams [b0, b0 + nbeam) of the B beams that G, w and bhat hold). This CTA
  // takes ti = blockIdx.x, blockIdx.x + gridDim.x, ...; every role walks the same sequence, and the
  // chunk counter gc runs on across tiles, so the rings never drain between tiles.
  auto tile_of = [&](int ti, int& m0, int& b, int& blk0) {
    m0 = (ti % mtiles) * kTileM;
    b = b0 + (ti / mtiles) % nbeam;
    blk0 = (ti / (mtiles * nbeam)) * NB;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < RS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&rawfree[s], 128);
    }
    for (int s = 0; s < PS; ++s) {
      mbar_init(&wconv[s], 128);
      mbar_init(&wfree[s], 1);
    }
    for (int k = 0; k < KSTEPS; ++k) {
      mbar_init(&aready[k], 128);
      mbar_init(&afree[k], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 128);
    mbar_init(mdone, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // Drain the accumulators of this CTA's tiles into bhat (tensor-memory lane quarter ew).
  auto epilogue = [&](int ew) {
    const uint32_t lane_base = tmem + ((uint32_t)(ew * 32) << 16);
    const bool two = nchunks >= 2;
    int it = 0;
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x, ++it) {
      int m0, b, blk0;
      tile_of(ti, m0, b, blk0);
      // Both exits are taken by the whole warp (the loop below shuffles across its lanes).
      const bool got = mbar_wait(tfull, it & 1, wait_ns);
      if (!__all_sync(0xffffffffu, got)) {
        if (lane == 0) atomicExch(status, (int)FBST_ERR_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int n = m0 + ew * 32 + lane;
      // FP16 split: undo the beam's scale of G and the blocks' scales of w (exact powers of two).
      // Lane l holds the inverse scales of blocks blk0 + l and blk0 + 32 + l.
      float ginv = 1.f, winv0 = 1.f, winv1 = 1.f;
      if constexpr (F16) {
        ginv = pow2f(-gexp[b]);
        if (blk0 + lane < nblk) winv0 = pow2f(-block_scale_exp(wmax, blk0 + lane));
        if (NB > 32 && blk0 + 32 + lane < nblk) winv1 = pow2f(-block_scale_exp(wmax, blk0 + 32 + lane));
      }
#pragma unroll 1
      for (int j0 = 0; j0 < NB; j0 += 16) {
        uint32_t h0r[16], h0i[16], lor[16], loi[16], h1r[16], h1i[16];
        tmem_ld16_async(lane_base + H0 + j0, h0r);
        tmem_ld16_async(lane_base + H0 + NB + j0, h0i);
        tmem_ld16_async(lane_base + LO + j0, lor);
        tmem_ld16_async(lane_base + LO + NB + j0, loi);
        if (two) {
          tmem_ld16_async(lane_base + H1 + j0, h1r);
          tmem_ld16_async(lane_base + H1 + NB + j0, h1i);
        }
        tmem_wait_ld();
        float re[16], im[16], t0[16], t1[16];
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          re[jj] = __uint_as_float(h0r[jj]) + (two ? __uint_as_float(h1r[jj]) : 0.f);
          im[jj] = __uint_as_float(h0i[jj]) + (two ? __uint_as_float(h1i[jj]) : 0.f);
          t0[jj] = __uint_as_float(lor[jj]);
          t1[jj] = __uint_as_float(loi[jj]);
        }
        if (j0 + 16 >= NB) {
          // Every accumulator column has been read: the next tile's MMAs may start.
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(tempty)) : "memory");
        }
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int blk = blk0 + j0 + jj;
          float sc = 1.f;
          if constexpr (F16) {
            const int c = j0 + jj;  // the same for every lane: no divergence in the shuffle
            sc = ginv * __shfl_sync(0xffffffffu, c < 32 ? winv0 : winv1, c & 31);
          }
          if (blk < nblk && n < N)
            bhat[((size_t)blk * B + b) * N + n] = make_float2((re[jj] + t0[jj]) * sc, (im[jj] + t1[jj]) * sc);
        }
      }
    }
  };

  if (threadIdx.x == 0) {
    // ---------------- TMA producer ----------------
    int gc = 0, issued = 0;
    bool ok = true;
    for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
      int m0, b, blk0;
      tile_of(ti, m0, b, blk0);
      for (int c = 0; c < nchunks; ++c, ++gc) {
        const int s = gc % RS;
        if ((gc >= RS && !mbar_wait(&rawfree[s], ((gc / RS) - 1) & 1, wait_ns)) || *abort_flag) {
          ok = false;
          break;
        }
        uint8_t* st = smem + s * SM::RAW_BYTES;
        mbar_expect_tx(&full[s], SM::RAW_BYTES);
        tma_load_3d(st, &mapA, &full[s], c * KELEM, m0, b * 2 + 0);
        tma_load_3d(st + SM::A_TILE, &mapA, &full[s], c * KELEM, m0, b * 2 + 1);
        tma_load_3d(st + 2 * SM::A_TILE, &mapW, &full[s], 2 * c * KELEM, b * w_beam_mul, blk0);
        tma_load_3d(st + 2 * SM::A_TILE + SM::W_BOX, &mapW, &full[s], 2 * c * KELEM + KELEM, b * w_beam_mul, blk0);
        issued = gc + 1;
      }
    }
    if (!ok) {
      atomicExch(status, (int)FBST_ERR_TIMEOUT);
      *abort_flag = 1;
    }
    // Copies still in flight must land before the CTA can leave (on the normal path these phases
    // have completed already and the waits return at once).
    for (int g = (issued > RS ? issued - RS : 0); g < issued; ++g) (void)mbar_wait(&full[g % RS], (g / RS) & 1, kDrainNs);
  } else if (threadIdx.x == 32) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t ID = make_idesc(F16 ? 0u : 2u, kTileM, 2 * NB, false);
    int gc = 0, it = 0;
    bool ok = true;
    for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x, ++it) {
      // The accumulators of the previous tile must have been read out.
      if (it >= 1 && !mbar_wait(tempty, (it - 1) & 1, wait_ns)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int c = 0; c < nchunks && ok; ++c, ++gc) {
        const int ps = gc % PS;
        if (!mbar_wait(&wconv[ps], (gc / PS) & 1, wait_ns)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t bh = smem_u32(smem + SM::PL_OFF + ps * 2 * SM::WPL), bl = bh + SM::WPL;
        const uint32_t hacc = tmem + ((c & 1) ? H1 : H0), lacc = tmem + LO;
#pragma unroll
        for (int k = 0; k < KSTEPS; ++k) {
          if (!mbar_wait(&aready[k], gc & 1, wait_ns)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a = tmem + RING + 32 * k;  // [hi_re | hi_im | lo_re | lo_im], 8 columns each
          // rows NB..3NB = [W_re | W_im] and rows 0..2NB = [-W_im | W_re] of the hi and lo planes;
          // a K step is 32 bytes of a row in both variants (8 TF32 or 16 FP16 values)
          const uint32_t hfirst = (c < 2 && k == 0) ? 0u : 1u, lfirst = (c == 0 && k == 0) ? 0u : 1u;
          if constexpr (F16) {
            const uint64_t h1 = smem_desc_sw64(bh + NB * SM::WROW + k * 32), h2 = smem_desc_sw64(bh + k * 32);
            const uint64_t l1 = smem_desc_sw64(bl + NB * SM::WROW + k * 32), l2 = smem_desc_sw64(bl + k * 32);
            mma_f16_ts(hacc, a + 0, h1, ID, hfirst);
            mma_f16_ts(hacc, a + 8, h2, ID, 1u);
            mma_f16_ts(lacc, a + 0, l1, ID, lfirst);
            mma_f16_ts(lacc, a + 8, l2, ID, 1u);
            mma_f16_ts(lacc, a + 16, h1, ID, 1u);
            mma_f16_ts(lacc, a + 24, h2, ID, 1u);
          } else {
            const uint64_t h1 = smem_desc_sw128(bh + NB * kRowBytes + k * 32), h2 = smem_desc_sw128(bh + k * 32);
            const uint64_t l1 = smem_desc_sw128(bl + NB * kRowBytes + k * 32), l2 = smem_desc_sw128(bl + k * 32);
            mma_tf32_ts(hacc, a + 0, h1, ID, hfirst);  // hi_re x [W_re | W_im]_hi
            mma_tf32_ts(hacc, a + 8, h2, ID, 1u);      // hi_im x [-W_im | W_re]_hi
            mma_tf32_ts(lacc, a + 0, l1, ID, lfirst);  // hi_re x lo
            mma_tf32_ts(lacc, a + 8, l2, ID, 1u);      // hi_im x lo
            mma_tf32_ts(lacc, a + 16, h1, ID, 1u);     // lo_re x hi
            mma_tf32_ts(lacc, a + 24, h2, ID, 1u);     // lo_im x hi
          }
          mma_commit(&afree[k]);
        }
        if (ok) mma_commit(&wfree[ps]);
      }
      if (ok) mma_commit(tfull);
    }
    if (!ok) {
      atomicExch(status, (int)FBST_ERR_TIMEOUT);
      *abort_flag = 1;
      mma_commit(tfull);   // releases an epilogue waiting for this tile (it then sees the abort flag)
    }
    // Every MMA this thread issued must have finished before tensor memory is released, whether or
    // not the epilogue read the last accumulators: a commit to a barrier of its own, waited for once.
    mma_commit(mdone);
    (void)mbar_wait(mdone, 0, kDrainNs);
  } else if (warp >= 4 && warp < 8) {
    // ---------------- converters ----------------
    const int ct = threadIdx.x - 128;  // A row and tensor-memory lane
    const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    int gc = 0;
    bool ok = true;
    for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
      // FP16 split: this tile's scale of G (its beam) and of the one w row (block) this thread
      // converts, row ct % NB of the tile's blocks.
      float gsc = 1.f, wsc = 1.f;
      if constexpr (F16) {
        int m0, b, blk0;
        tile_of(ti, m0, b, blk0);
        gsc = pow2f(gexp[b]);
        if (blk0 + ct % NB < nblk) wsc = pow2f(block_scale_exp(wmax, blk0 + ct % NB));
      }
      for (int c = 0; c < nchunks; ++c, ++gc) {
        const int s = gc % RS, ps = gc % PS;
        if (!mbar_wait(&full[s], (gc / RS) & 1, wait_ns) || *abort_flag) {
          ok = false;
          break;
        }
        const uint8_t* raw = smem + s * SM::RAW_BYTES;
        // This thread's row of G for the whole chunk: 16-byte chunk j of row ct sits at j ^ (ct & 7).
        float4 ar[KELEM / 4], ai[KELEM / 4];
#pragma unroll
        for (int j = 0; j < KELEM / 4; ++j) {
          const int off = ct * kRowBytes + ((j ^ (ct & 7)) << 4);
          ar[j] = *reinterpret_cast<const float4*>(raw + off);
          ai[j] = *reinterpret_cast<const float4*>(raw + SM::A_TILE + off);
        }
        if (gc >= PS && !mbar_wait(&wfree[ps], ((gc / PS) - 1) & 1, wait_ns)) {
          ok = false;
          break;
        }
        uint8_t* ph = smem + SM::PL_OFF + ps * 2 * SM::WPL;
        if constexpr (F16) {
          // B: 8 complex values (64 raw bytes) -> one 16-byte chunk (row r, chunk q of 4) of the -W_im,
          // W_re and W_im rows of both FP16 planes, 64-byte swizzle. The raw boxes arrive in the
          // 128-byte swizzle (16-byte chunk c of row r at c ^ (r & 7)) and consecutive threads take
          // consecutive rows, so the 8 threads of a quarter warp read and write 8 different bank
          // groups. Every item of this thread is in row ct % NB.
#pragma unroll 2
          for (int j = ct; j < NB * 4; j += 128) {
            const int r = j % NB, q = j / NB;
            const uint8_t* rp = raw + 2 * SM::A_TILE + (q >> 1) * SM::W_BOX + r * kRowBytes;
            float4 x[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
              x[i] = *reinterpret_cast<const float4*>(rp + ((((q & 1) * 4 + i) ^ (r & 7)) << 4));
            const float sc = wsc;
            uint32_t rh[4], ih[4], nih[4], rl[4], il[4], nil[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float re0 = x[i].x * sc, im0 = x[i].y * sc, re1 = x[i].z * sc, im1 = x[i].w * sc;
              const __half2 hr = __floats2half2_rn(re0, re1), hi2 = __floats2half2_rn(im0, im1);
              const __half2 lr = __floats2half2_rn(re0 - __low2float(hr), re1 - __high2float(hr));
              const __half2 li = __floats2half2_rn(im0 - __low2float(hi2), im1 - __high2float(hi2));
              rh[i] = h2_bits(hr);
              ih[i] = h2_bits(hi2);
              nih[i] = ih[i] ^ 0x80008000u;
              rl[i] = h2_bits(lr);
              il[i] = h2_bits(li);
              nil[i] = il[i] ^ 0x80008000u;
            }
            const int off = r * SM::WROW + ((q ^ ((r >> 1) & 3)) << 4);
            uint8_t* hp = ph + off;
            uint8_t* lp = ph + SM::WPL + off;
            *reinterpret_cast<uint4*>(hp) = make_uint4(nih[0], nih[1], nih[2], nih[3]);
            *reinterpret_cast<uint4*>(hp + NB * SM::WROW) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
            *reinterpret_cast<uint4*>(hp + 2 * NB * SM::WROW) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
            *reinterpret_cast<uint4*>(lp) = make_uint4(nil[0], nil[1], nil[2], nil[3]);
            *reinterpret_cast<uint4*>(lp + NB * SM::WROW) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
            *reinterpret_cast<uint4*>(lp + 2 * NB * SM::WROW) = make_uint4(il[0], il[1], il[2], il[3]);
          }
        } else {
        // B: 4 complex values (32 raw bytes) -> one 16-byte chunk (row r, chunk q) of the -W_im, W_re
        // and W_im rows of both planes, at the swizzled position. The two raw halves are read in an
        // order that depends on the box, so the 8 threads of one row touch 8 different bank groups.
#pragma unroll 2
        for (int j = ct; j < NB * 8; j += 128) {
          const int r = j >> 3, q = j & 7, box = q >> 2;
          const uint8_t* rp = raw + 2 * SM::A_TILE + box * SM::W_BOX + r * kRowBytes + (q & 3) * 32;
          const float4 x0 = *reinterpret_cast<const float4*>(rp + 16 * box);
          const float4 x1 = *reinterpret_cast<const float4*>(rp + 16 * (1 - box));
          const float4 a = box ? x1 : x0, bb = box ? x0 : x1;
          const float4 re = make_float4(a.x, a.z, bb.x, bb.z), im = make_float4(a.y, a.w, bb.y, bb.w);
          const float4 rh = rna4(re), ih = rna4(im), rl = sub4(re, rh), il = sub4(im, ih);
          const int off = r * kRowBytes + ((q ^ (r & 7)) << 4);
          uint8_t* hp = ph + off;
          uint8_t* lp = ph + SM::WPL + off;
          *reinterpret_cast<float4*>(hp) = neg4(ih);
          *reinterpret_cast<float4*>(hp + NB * kRowBytes) = rh;
          *reinterpret_cast<float4*>(hp + 2 * NB * kRowBytes) = ih;
          *reinterpret_cast<float4*>(lp) = neg4(il);
          *reinterpret_cast<float4*>(lp + NB * kRowBytes) = rl;
          *reinterpret_cast<float4*>(lp + 2 * NB * kRowBytes) = il;
        }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&wconv[ps])) : "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&rawfree[s])) : "memory");
        // A: split each K step into tensor-memory slot k once the MMAs of the previous chunk freed it.
#pragma unroll
        for (int k = 0; k < KSTEPS; ++k) {
          uint32_t hi[16], lo[16];
          if constexpr (F16) {
            // K step k = 16 values per plane (float4s 4k..4k+3); column c holds values 2c, 2c+1.
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const float4* src = e ? ai : ar;
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const float4 v = src[4 * k + i];
                const float a0 = v.x * gsc, a1 = v.y * gsc, a2 = v.z * gsc, a3 = v.w * gsc;
                const __half2 h01 = __floats2half2_rn(a0, a1), h23 = __floats2half2_rn(a2, a3);
                hi[e * 8 + 2 * i] = h2_bits(h01);
                hi[e * 8 + 2 * i + 1] = h2_bits(h23);
                lo[e * 8 + 2 * i] = h2_bits(__floats2half2_rn(a0 - __low2float(h01), a1 - __high2float(h01)));
                lo[e * 8 + 2 * i + 1] = h2_bits(__floats2half2_rn(a2 - __low2float(h23), a3 - __high2float(h23)));
              }
            }
          } else {
            const float x[2][8] = {{ar[2 * k].x, ar[2 * k].y, ar[2 * k].z, ar[2 * k].w, ar[2 * k + 1].x,
                                    ar[2 * k + 1].y, ar[2 * k + 1].z, ar[2 * k + 1].w},
                                   {ai[2 * k].x, ai[2 * k].y, ai[2 * k].z, ai[2 * k].w, ai[2 * k + 1].x,
                                    ai[2 * k + 1].y, ai[2 * k + 1].z, ai[2 * k + 1].w}};
#pragma unroll
            for (int e = 0; e < 2; ++e) {
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const float h = round_tf32(x[e][i]);
                hi[e * 8 + i] = __float_as_uint(h);
                lo[e * 8 + i] = __float_as_uint(x[e][i] - h);
              }
            }
          }
          if (gc >= 1 && !mbar_wait(&afree[k], (gc - 1) & 1, wait_ns)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          tmem_st16(lane_addr + RING + 32 * k, hi);
          tmem_st16(lane_addr + RING + 32 * k + 16, lo);
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&aready[k])) : "memory");
        }
        if (!ok) break;
      }
    }
    if (!ok && lane == 0) {
      atomicExch(status, (int)FBST_ERR_TIMEOUT);
      *abort_flag = 1;
    }
  } else if (PERSIST && warp >= 8) {
    epilogue(warp & 3);
  }
  __syncwarp();
  // A single-tile CTA has no epilogue warps: warps 0-3 drain the accumulators after the main loop.
  if constexpr (!PERSIST) {
    if (warp < 4) epilogue(warp);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// G [B][N][L] complex64 -> FP32 planes [B][2][N][L] (real, imaginary).
__global__ void k_tc_planes_f32(const float2* __restrict__ G, float* __restrict__ out, int B, int N, int L) {
  const size_t per_beam = (size_t)N * L;
  const size_t total = (size_t)B * per_beam;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / per_beam, r = i % per_beam;
    const float2 g = G[i];
    out[(b * 2 + 0) * per_beam + r] = g.x;
    out[(b * 2 + 1) * per_beam + r] = g.y;
  }
}

// Largest magnitude of any real or imaginary part of beam b's G planes ([2][N][L] FP32) ->
// gexp[b], the exponent of the beam's FP16 scale (one CTA per beam).
__global__ void k_tc_gexp(const float* __restrict__ planes, int* __restrict__ gexp, size_t per_beam) {
  const float4* src = reinterpret_cast<const float4*>(planes + (size_t)blockIdx.x * per_beam);
  float m = 0.f;
  for (size_t i = threadIdx.x; i < per_beam / 4; i += blockDim.x) {
    const float4 v = src[i];
    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) gexp[blockIdx.x] = scale_exp(m);
  }
}

// Largest |re|, |im| over block blk of w (rows x 2L floats, contiguous per block): kWParts CTAs per
// block, each over an equal float4 range, combine by atomicMax on the float bits into wmax[blk]
// (zeroed first; the maximum does not depend on the order).
__global__ void k_tc_wmax(const float* __restrict__ w, unsigned* __restrict__ wmax, size_t per_block4) {
  const int blk = blockIdx.y, part = blockIdx.x;
  const float4* src = reinterpret_cast<const float4*>(w) + (size_t)blk * per_block4;
  const size_t i0 = per_block4 * part / kWParts, i1 = per_block4 * (part + 1) / kWParts;
  float m = 0.f;
  for (size_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const float4 v = src[i];
    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) atomicMax(wmax + blk, __float_as_uint(m));
  }
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 3-D map over planes [Z][Y][X] (X contiguous, ESZ-byte elements), box {128 bytes of X, boxY, 1},
// 128-byte swizzle; out-of-range elements read as zero.
static int make_map(CUtensorMap* map, const void* base, int esz, uint64_t X, uint64_t Y, uint64_t Z, uint32_t boxY) {
  auto enc = tensor_map_encoder();
  if (!enc) return FBST_ERR_UNSUPPORTED;
  const cuuint64_t dims[3] = {X, Y, Z};
  const cuuint64_t strides[2] = {X * esz, X * Y * esz};
  const cuuint32_t box[3] = {(cuuint32_t)(kRowBytes / esz), boxY, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType dt = esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const CUresult r = enc(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? FBST_OK : FBST_ERR_CUDA;
}

// 3-D map over the interleaved complex64 w [nblk][B][L] read as floats: dims {2L, B, nblk}, box
// {32 floats, 1, boxZ}; no swizzle for the TF32 split (its converter warps index it themselves), the
// 128-byte swizzle for the FP16 split.
static int make_map_w(CUtensorMap* map, const void* base, uint64_t L2f, uint64_t B, uint64_t nblk, uint32_t boxZ,
                      bool swizzle128 = false) {
  auto enc = tensor_map_encoder();
  if (!enc) return FBST_ERR_UNSUPPORTED;
  const cuuint64_t dims[3] = {L2f, B, nblk};
  const cuuint64_t strides[2] = {L2f * 4, L2f * B * 4};
  const cuuint32_t box[3] = {(cuuint32_t)(kRowBytes / 4), 1, boxZ};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE,
                         swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? FBST_OK : FBST_ERR_CUDA;
}

template <int V>
static size_t plane_bytes_G(const fbst_info& in) {
  return (size_t)in.B * tc_traits<V>::NPL * in.N * in.L * tc_traits<V>::ESZ;
}

static int round16(int x) { return (x + 15) / 16 * 16; }

template <int V>
static int build_operand_V(fbst_plan_s* p, cudaStream_t s) {
  const fbst_info& in = p->info;
  if (in.L % 8 != 0) return FBST_ERR_UNSUPPORTED;  // 16-byte rows for TMA
  const size_t bytes = plane_bytes_G<V>(in);
  FBST_TRY(plan_alloc(p, bytes, &p->Gtc));
  p->Gtc_bytes = bytes;
  k_tc_split_G<V><<<4096, 256, 0, s>>>(p->G, p->Gtc, in.B, in.N, in.L);
  FBST_CUDA_TRY(cudaGetLastError());
  const int NBW = round16(p->band.max_blocks);
  p->ws_tc_bytes = (size_t)in.B * tc_traits<V>::NPL * NBW * in.L * tc_traits<V>::ESZ;
  FBST_TRY(plan_alloc(p, p->ws_tc_bytes, &p->ws_tc));
  FBST_CUDA_TRY(cudaMemsetAsync(p->ws_tc, 0, p->ws_tc_bytes, s));
  return FBST_OK;
}

static int build_operand_fused(fbst_plan_s* p, bool f16, cudaStream_t s) {
  const fbst_info& in = p->info;
  if (in.L % 8 != 0) return FBST_ERR_UNSUPPORTED;
  const size_t bytes = (size_t)in.B * 2 * in.N * in.L * sizeof(float);
  FBST_TRY(plan_alloc(p, bytes, &p->Gtc));
  p->Gtc_bytes = bytes;
  k_tc_planes_f32<<<4096, 256, 0, s>>>(p->G, static_cast<float*>(p->Gtc), in.B, in.N, in.L);
  FBST_CUDA_TRY(cudaGetLastError());
  if (f16) {
    // The FP16 split scales each beam's G and each block's w by a power of two.
    FBST_TRY(plan_alloc_n(p, &p->tc_gexp, (size_t)in.B));
    FBST_TRY(plan_alloc_n(p, &p->tc_wmax, (size_t)p->band.max_blocks));
    // The spatial chirp-z of a linear grid array finds the block maxima as it writes w.
    p->tc_wmax_stage1 = p->geom.kind == FBST_ULA && !p->nu_nf;
    k_tc_gexp<<<in.B, 256, 0, s>>>(static_cast<const float*>(p->Gtc), p->tc_gexp, (size_t)2 * in.N * in.L);
    FBST_CUDA_TRY(cudaGetLastError());
  }
  return FBST_OK;
}

int build_dense_tc_operand(fbst_plan_s* p, cudaStream_t s) {
  if (!tensor_map_encoder()) return FBST_ERR_UNSUPPORTED;
  switch (variant_of(p->info.stage2)) {
    case TC_BF16X3: return build_operand_V<TC_BF16X3>(p, s);
    case TC_TF32: return build_operand_V<TC_TF32>(p, s);
    case TC_TF32X3: return build_operand_fused(p, false, s);
    case TC_F16X3: return build_operand_fused(p, true, s);
    default: return FBST_ERR_INVALID;
  }
}

template <int V, int NB>
static int gemm_NB(const fbst_plan_s* p, float2* bhat, int nblk, cudaStream_t s) {
  using TR = tc_traits<V>;
  const fbst_info& in = p->info;
  const int NBW = round16(p->band.max_blocks);
  CUtensorMap mapA, mapB;
  int r = make_map(&mapA, p->Gtc, TR::ESZ, in.L, in.N, (uint64_t)in.B * TR::NPL, kTileM);
  if (r != FBST_OK) return r;
  r = make_map(&mapB, p->ws_tc, TR::ESZ, in.L, NBW, (uint64_t)in.B * TR::NPL, NB);
  if (r != FBST_OK) return r;
  const int smem = tc_smem<V, NB>::BYTES;
  FBST_CUDA_TRY(cudaFuncSetAttribute(k_dense_tc<V, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const dim3 grid((in.N + kTileM - 1) / kTileM, in.B, (nblk + NB - 1) / NB);
  k_dense_tc<V, NB><<<grid, 128, smem, s>>>(mapA, mapB, bhat, in.B, in.N, in.L, nblk, p->d_status,
                                            p->wait_ns ? p->wait_ns : kWaitNs);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

template <int V>
static int launch_V(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk, cudaStream_t s) {
  using TR = tc_traits<V>;
  const fbst_info& in = p->info;
  const int NBW = round16(p->band.max_blocks);
  const int nrows = round16(nblk);
  if (nrows > NBW) return FBST_ERR_INVALID;
  k_tc_prep_w<V><<<dim3(std::min(64, (nrows * in.L + 255) / 256), in.B), 256, 0, s>>>(w, p->ws_tc, in.B, in.L, nblk,
                                                                                     nrows, NBW);
  FBST_CUDA_TRY(cudaGetLastError());
  // Smallest MMA width that covers the blocks (16..MAX_NB in steps of 16).
  const int want = std::min(nrows, TR::MAX_NB);
  if (want <= 16) return gemm_NB<V, 16>(p, bhat, nblk, s);
  if (want <= 32) return gemm_NB<V, 32>(p, bhat, nblk, s);
  if (want <= 64) return gemm_NB<V, 64>(p, bhat, nblk, s);
  if constexpr (TR::MAX_NB >= 128) return gemm_NB<V, 128>(p, bhat, nblk, s);
  return FBST_ERR_INVALID;
}

template <int NB, bool F16>
static int gemm_fused(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk, int b0, int nbeam,
                      bool shared_rhs, cudaStream_t s) {
  const fbst_info& in = p->info;
  CUtensorMap mapA, mapW;
  int r = make_map(&mapA, p->Gtc, 4, in.L, in.N, (uint64_t)in.B * 2, kTileM);
  if (r != FBST_OK) return r;
  // A shared right-hand side is one row per block that every beam reads (beam coordinate 0).
  r = make_map_w(&mapW, w, 2 * (uint64_t)in.L, shared_rhs ? 1 : in.B, nblk, NB, F16);
  if (r != FBST_OK) return r;
  // NB >= 32: one CTA per SM is all that shared and tensor memory allow, so it is persistent and
  // walks its tiles. NB = 16: two single-tile CTAs (256 threads, 256 tensor-memory columns) fit
  // on an SM, which keeps more of G in flight than one persistent CTA does.
  constexpr bool kPersist = NB >= 32;
  const int smem = fused_smem<NB, F16>::BYTES;
  FBST_CUDA_TRY(cudaFuncSetAttribute(k_dense_tc_fused<NB, kPersist, F16>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const long long ntiles = (long long)((in.N + kTileM - 1) / kTileM) * nbeam * ((nblk + NB - 1) / NB);
  if (ntiles > INT_MAX) return FBST_ERR_UNSUPPORTED;
  const int grid = kPersist ? (int)std::min<long long>(ntiles, sm_count()) : (int)ntiles;
  k_dense_tc_fused<NB, kPersist, F16><<<grid, kPersist ? 384 : 256, smem, s>>>(
      mapA, mapW, bhat, in.B, in.N, in.L, nblk, b0, nbeam, shared_rhs ? 0 : 1, p->tc_gexp, p->tc_wmax,
      p->d_status, p->wait_ns ? p->wait_ns : kWaitNs);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

template <bool F16>
static int launch_fused_F(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk, int b0, int nbeam,
                          cudaStream_t s, bool shared_rhs) {
  const int want = std::min(round16(nblk), 64);
  if (want <= 16) return gemm_fused<16, F16>(p, w, bhat, nblk, b0, nbeam, shared_rhs, s);
  if (want <= 32) return gemm_fused<32, F16>(p, w, bhat, nblk, b0, nbeam, shared_rhs, s);
  return gemm_fused<64, F16>(p, w, bhat, nblk, b0, nbeam, shared_rhs, s);
}

static int launch_fused(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk, int b0, int nbeam,
                        cudaStream_t s, bool shared_rhs = false) {
  if (variant_of(p->info.stage2) == TC_F16X3) return launch_fused_F<true>(p, w, bhat, nblk, b0, nbeam, s, shared_rhs);
  return launch_fused_F<false>(p, w, bhat, nblk, b0, nbeam, s, shared_rhs);
}

static bool fused_variant(const fbst_plan_s* p) {
  const int v = variant_of(p->info.stage2);
  return v == TC_TF32X3 || v == TC_F16X3;
}

int prepare_dense_tc_scales(const fbst_plan_s* p, const float2* w, int nblk, cudaStream_t s) {
  if (variant_of(p->info.stage2) != TC_F16X3 || nblk <= 0) return FBST_OK;
  if (!p->tc_wmax || nblk > p->band.max_blocks || nblk > 65535) return FBST_ERR_INVALID;
  const size_t per_block4 = (size_t)p->info.B * p->info.L / 2;  // B x L complex64 = B L / 2 float4
  FBST_CUDA_TRY(cudaMemsetAsync(p->tc_wmax, 0, sizeof(unsigned) * nblk, s));
  k_tc_wmax<<<dim3(kWParts, nblk), 256, 0, s>>>(reinterpret_cast<const float*>(w), p->tc_wmax, per_block4);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

int launch_dense_tc_shared_rhs(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk, cudaStream_t s) {
  if (variant_of(p->info.stage2) != TC_TF32X3) return FBST_ERR_UNSUPPORTED;
  if (nblk <= 0) return FBST_OK;
  if (!p->Gtc) return FBST_ERR_INVALID;
  return launch_fused(p, w, bhat, nblk, 0, p->info.B, s, true);
}

int launch_stage2_dense_tc_beams(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk, int b0, int nbeam,
                                 cudaStream_t s) {
  if (!fused_variant(p)) return FBST_ERR_UNSUPPORTED;
  if (b0 < 0 || nbeam < 0 || b0 + nbeam > p->info.B) return FBST_ERR_INVALID;
  if (nblk <= 0 || nbeam == 0) return FBST_OK;
  if (!p->Gtc) return FBST_ERR_INVALID;
  return launch_fused(p, w, bhat, nblk, b0, nbeam, s);
}

int launch_stage2_dense_tc(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk, cudaStream_t s,
                           bool scales_ready) {
  if (nblk <= 0) return FBST_OK;
  if (!p->Gtc) return FBST_ERR_INVALID;
  if (fused_variant(p)) {
    if (!scales_ready) FBST_TRY(prepare_dense_tc_scales(p, w, nblk, s));
    return launch_fused(p, w, bhat, nblk, 0, p->info.B, s);
  }
  if (!p->ws_tc) return FBST_ERR_INVALID;
  switch (variant_of(p->info.stage2)) {
    case TC_BF16X3: return launch_V<TC_BF16X3>(p, w, bhat, nblk, s);
    case TC_TF32: return launch_V<TC_TF32>(p, w, bhat, nblk, s);
    default: return FBST_ERR_INVALID;
  }
}

}  // namespace fbst
