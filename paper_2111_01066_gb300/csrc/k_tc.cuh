// Complex GEMM on the fifth-generation tensor cores (tcgen05, sm_103a).
//
// C[m, n] = sum_k A[m, k] B[k, n] (SI, Eq. (2)) as ONE real GEMM per tile:
//   D[m, (n, t)] = sum_{(k, u)} A'[m, (k, u)] B'[(n, t), (k, u)]
// with A'[m, (k, 0)] = Re A, A'[m, (k, 1)] = Im A (the interleaved complex64
// storage itself), and the 2x2 real form of every B entry:
//   B'[(n,0),(k,0)] = Re B, B'[(n,0),(k,1)] = -Im B, B'[(n,1),(k,0)] = Im B,
//   B'[(n,1),(k,1)] = Re B,
// so that D[m, (n,0)] = Re C and D[m, (n,1)] = Im C: the accumulator rows are
// interleaved complex64 rows of C.  Four real products per complex product (4M).
//
// Precision modes: TF32 (kind::tf32, one MMA per K step) and BF16X3
// (kind::f16 with bf16 hi/lo split operands: hi*hi + hi*lo + lo*hi, FP32
// accumulation in TMEM).
//
// A (the large, streamed operand) is gathered by loader warps straight from
// its tensor's storage order -- the index permutation of Eq. (2) is folded into
// the loads, as in the paper's fused permutation-multiplication (SI, figure
// S7a).  B' (small) is written once per step by k_tc_prep_b in the exact
// shared-memory image of every (n tile, k chunk) and fetched by one bulk copy.
//
// Roles (416 threads, one CTA per SM, persistent over tiles):
//   warps 0-3  epilogue: TMEM -> registers -> C (lane = tile row)
//   warp  4    TMEM allocation; lane 0 issues tcgen05.mma and commits
//   warps 5-12 loaders: A gathers + B' bulk copy per pipeline stage
// Every mbarrier wait is bounded by a globaltimer deadline; on expiry the
// kernel records TN_ERR_TIMEOUT in *err, every role leaves its loop, and the
// CTA frees its TMEM and returns.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels_common.cuh"

namespace tnx {

constexpr int TC_M = 128;
constexpr int TC_TK = 16;            // complex k per pipeline stage
constexpr int TC_KP = 2 * TC_TK;     // real K' per stage
constexpr int TC_STAGES = 4;
constexpr int TC_EPI_WARPS = 4;
constexpr int TC_MMA_WARP = 4;
constexpr int TC_LOAD_WARPS = 8;
constexpr int TC_LOAD_THREADS = TC_LOAD_WARPS * 32;
constexpr int TC_THREADS = (TC_EPI_WARPS + 1 + TC_LOAD_WARPS) * 32;
constexpr int TC_AE = TC_M * TC_TK / TC_LOAD_THREADS;    // A elements per loader thread per stage
constexpr int TC_TMEM_COLS = 512;
constexpr uint64_t TC_WAIT_NS = 4000000000ull;           // 4 s per wait
constexpr int TC_MIN_SMEM = 120 * 1024;                  // keeps one CTA per SM

enum TcMode { TC_TF32 = 0, TC_BF16X3 = 1 };

template <int MODE>
struct TcT;
template <>
struct TcT<TC_TF32> {
  static constexpr int ESZ = 4, NPL = 1, FMT = 2;
};
template <>
struct TcT<TC_BF16X3> {
  static constexpr int ESZ = 2, NPL = 2, FMT = 1;
};

// bytes of one operand plane per stage: rows x 32 real elements
__host__ __device__ constexpr int tc_plane_bytes(int rows, int esz) { return rows * TC_KP * esz; }
// 16-byte chunks per row of one plane, and the stride between 8-row groups
__host__ __device__ constexpr int tc_cpr(int esz) { return TC_KP * esz / 16; }
__host__ __device__ constexpr int tc_sbo(int esz) { return tc_cpr(esz) * 128; }
// byte offset of real element (row, kp) inside a K-major no-swizzle plane
__host__ __device__ inline int tc_elem_off(int row, int kp, int esz) {
  const int byte = kp * esz;
  return (row >> 3) * tc_sbo(esz) + (byte >> 4) * 128 + (row & 7) * 16 + (byte & 15);
}

struct TcArgs {
  GemmArgs g;
  const uint8_t* bimg;   // B' images, [inst][n tile][k chunk] blocks
  int32_t tn_c;          // complex columns per tile (>= 8); N' = 2 tn_c
  int32_t tnb;           // n bits covered by a tile (valid columns = 2^tnb)
  int32_t n_mt, n_nt, n_kc;
  int64_t n_tiles;
  int32_t* err;
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: true when the phase completed, false on abort or deadline.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag,
                                          int32_t* err) {
  if (mbar_try_wait(a, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(a, parity)) return true;
    if ((i & 255) == 0) {
      if (*abort_flag) return false;
      if (gtimer() - t0 > TC_WAIT_NS) {
        *abort_flag = 1;
        atomicExch(err, TN_ERR_TIMEOUT);
        return false;
      }
    }
  }
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive_noinc(uint32_t mbar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}
// shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;
}
template <int MODE>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  if constexpr (MODE == TC_TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo_elem, float hi_elem) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo_elem, hi_elem);
  return *reinterpret_cast<uint32_t*>(&h);
}

// ------------------------------------------------------------------ B' images
// One thread per complex B entry of every (instance, n tile, k chunk) block;
// writes its 2x2 real form (split into hi/lo for BF16X3) at its place in the
// block's shared-memory image.  Padding (k or n beyond the operand) is zero.
template <int MODE>
__global__ void k_tc_prep_b(const TcArgs a) {
  using T = TcT<MODE>;
  const GemmArgs& g = a.g;
  const int ncp = 2 * a.tn_c;
  const int plane = tc_plane_bytes(ncp, T::ESZ);
  const int64_t block_bytes = (int64_t)T::NPL * plane;
  const int per_block = TC_TK * a.tn_c;
  const int64_t total = (int64_t)g.n_inst * a.n_nt * a.n_kc * per_block;
  const int tkv = 1 << g.tk, tnv = 1 << a.tnb;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(idx % per_block);
    const int64_t blk = idx / per_block;
    const int kc = (int)(blk % a.n_kc);
    const int nt = (int)((blk / a.n_kc) % a.n_nt);
    const int inst = (int)(blk / ((int64_t)a.n_kc * a.n_nt));
    const int kl = e % TC_TK, nl = e / TC_TK;
    float2 b = make_float2(0.f, 0.f);
    if (kl < tkv && nl < tnv) {
      const int64_t off = inst_offset(inst, g.b_istride, g.b_bpos, g.nb) +
                          deposit_hi((uint64_t)kl, g.b_kpos, 0, g.tk) +
                          deposit_hi((uint64_t)kc, g.b_kpos, g.tk, g.nk) +
                          deposit_hi((uint64_t)nl, g.b_npos, 0, a.tnb) +
                          deposit_hi((uint64_t)nt, g.b_npos, a.tnb, g.nn);
      b = g.B[off];
    }
    uint8_t* base = const_cast<uint8_t*>(a.bimg) + blk * block_bytes;
    // rows (n, t), columns (k, u)
    const float v[2][2] = {{b.x, -b.y}, {b.y, b.x}};
    for (int t = 0; t < 2; ++t)
      for (int u = 0; u < 2; ++u) {
        const int row = 2 * nl + t, kp = 2 * kl + u;
        const int off = tc_elem_off(row, kp, T::ESZ);
        if constexpr (MODE == TC_TF32) {
          uint32_t bits;
          asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(bits) : "f"(v[t][u]));
          *reinterpret_cast<uint32_t*>(base + off) = bits;
        } else {
          const __nv_bfloat16 hi = __float2bfloat16_rn(v[t][u]);
          const __nv_bfloat16 lo = __float2bfloat16_rn(v[t][u] - __bfloat162float(hi));
          *reinterpret_cast<__nv_bfloat16*>(base + off) = hi;
          *reinterpret_cast<__nv_bfloat16*>(base + plane + off) = lo;
        }
      }
  }
}

// ------------------------------------------------------------------ the GEMM
template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1) k_cgemm_tc(const TcArgs a) {
  using T = TcT<MODE>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const GemmArgs& g = a.g;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncp = 2 * a.tn_c;                                   // N'
  const int a_plane = tc_plane_bytes(TC_M, T::ESZ);
  const int b_plane = tc_plane_bytes(ncp, T::ESZ);
  const int stage_bytes = T::NPL * (a_plane + b_plane);
  uint8_t* stages = smem_raw;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + TC_STAGES * stage_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + TC_STAGES;
  uint64_t* tfull = bars + 2 * TC_STAGES;
  uint64_t* tempty = bars + 2 * TC_STAGES + 2;
  uint64_t* fin = bars + 2 * TC_STAGES + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * TC_STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int64_t* offCm = reinterpret_cast<int64_t*>(tmem_slot + 4);
  int64_t* offCn = offCm + TC_M;

  // zero every stage once: padding rows / columns are never written again
  for (int i = threadIdx.x; i < TC_STAGES * stage_bytes / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(stages)[i] = make_uint4(0, 0, 0, 0);
  const int tmv = 1 << g.tm, tnv = 1 << a.tnb;
  for (int r = threadIdx.x; r < TC_M; r += blockDim.x)
    offCm[r] = r < tmv ? deposit_hi((uint64_t)r, g.c_mpos, 0, g.tm) : 0;
  for (int c = threadIdx.x; c < 128; c += blockDim.x)
    offCn[c] = c < tnv ? deposit_hi((uint64_t)c, g.c_npos, 0, a.tnb) : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), TC_LOAD_THREADS);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&tfull[i]), 1);
      mbar_init(smem_u32(&tempty[i]), TC_EPI_WARPS * 32);
    }
    mbar_init(smem_u32(fin), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == TC_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int kc_n = a.n_kc;

  if (warp >= TC_MMA_WARP + 1) {
    // ---------------------------------------------------------------- loaders
    const int lt = threadIdx.x - (TC_MMA_WARP + 1) * 32;
    // decode this thread's tile elements once: (smem offset, gmem offset)
    int sm_off[TC_AE];
    int64_t gm_off[TC_AE];
    const int a_elems = 1 << g.a_tbits;
#pragma unroll
    for (int j = 0; j < TC_AE; ++j) {
      const int e = lt + j * TC_LOAD_THREADS;
      sm_off[j] = -1;
      gm_off[j] = 0;
      if (e < a_elems) {
        int r = 0, c = 0;
        int64_t off = 0;
        for (int t = 0; t < g.a_tbits; ++t)
          if ((e >> t) & 1) {
            const int s = g.a_tsel[t];
            if (s & 64) c |= 1 << (s & 63); else r |= 1 << (s & 63);
            off += (int64_t)1 << g.a_tpos[t];
          }
        sm_off[j] = tc_elem_off(r, 2 * c, T::ESZ);
        gm_off[j] = off;
      }
    }
    int stage = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < a.n_tiles && ok; tile += gridDim.x) {
      const int nt = (int)(tile % a.n_nt);
      const int64_t rest = tile / a.n_nt;
      const int mt = (int)(rest % a.n_mt);
      const int inst = (int)(rest / a.n_mt);
      const float2* A = g.A + inst_offset(inst, g.a_istride, g.a_bpos, g.nb) +
                        deposit_hi((uint64_t)mt, g.a_mpos, g.tm, g.nm);
      const uint8_t* bsrc = a.bimg + ((int64_t)inst * a.n_nt + nt) * (int64_t)kc_n * (T::NPL * b_plane);
      for (int kc = 0; kc < kc_n; ++kc) {
        const float2* Ak = A + deposit_hi((uint64_t)kc, g.a_kpos, g.tk, g.nk);
        uint8_t* sa = stages + stage * stage_bytes;
        uint8_t* sb = sa + T::NPL * a_plane;
        const uint32_t fb = smem_u32(&full[stage]);
        if constexpr (MODE == TC_TF32) {
          if (!mbar_wait(smem_u32(&empty[stage]), ph ^ 1, abort_flag, a.err)) { ok = false; break; }
          if (lt == 0) {
            mbar_expect_tx(fb, (uint32_t)(T::NPL * b_plane));
            bulk_g2s(smem_u32(sb), bsrc + (int64_t)kc * (T::NPL * b_plane), T::NPL * b_plane, fb);
          }
#pragma unroll
          for (int j = 0; j < TC_AE; ++j)
            if (sm_off[j] >= 0) cp_async8(smem_u32(sa + sm_off[j]), Ak + gm_off[j]);
          cp_async_arrive_noinc(fb);
        } else {
          float2 v[TC_AE];
#pragma unroll
          for (int j = 0; j < TC_AE; ++j)
            if (sm_off[j] >= 0) v[j] = __ldg(Ak + gm_off[j]);
          if (!mbar_wait(smem_u32(&empty[stage]), ph ^ 1, abort_flag, a.err)) { ok = false; break; }
          if (lt == 0) {
            mbar_expect_tx(fb, (uint32_t)(T::NPL * b_plane));
            bulk_g2s(smem_u32(sb), bsrc + (int64_t)kc * (T::NPL * b_plane), T::NPL * b_plane, fb);
          }
#pragma unroll
          for (int j = 0; j < TC_AE; ++j)
            if (sm_off[j] >= 0) {
              const __nv_bfloat162 hi = __floats2bfloat162_rn(v[j].x, v[j].y);
              const float2 hf = __bfloat1622float2(hi);
              const __nv_bfloat162 lo = __floats2bfloat162_rn(v[j].x - hf.x, v[j].y - hf.y);
              *reinterpret_cast<__nv_bfloat162*>(sa + sm_off[j]) = hi;
              *reinterpret_cast<__nv_bfloat162*>(sa + a_plane + sm_off[j]) = lo;
            }
          fence_proxy_async();
          mbar_arrive(fb);
        }
        if (++stage == TC_STAGES) {
          stage = 0;
          ph ^= 1;
        }
      }
    }
    if constexpr (MODE == TC_TF32) asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp == TC_MMA_WARP) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | ((uint32_t)T::FMT << 7) | ((uint32_t)T::FMT << 10) |
                             ((uint32_t)(ncp >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
      const uint32_t sbo = tc_sbo(T::ESZ);
      int stage = 0;
      uint32_t ph = 0;
      int64_t it = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < a.n_tiles && ok; tile += gridDim.x, ++it) {
        const int acc = (int)(it & 1);
        const uint32_t aph = (uint32_t)((it >> 1) & 1);
        if (!mbar_wait(smem_u32(&tempty[acc]), aph ^ 1, abort_flag, a.err)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * ncp);
        for (int kc = 0; kc < kc_n; ++kc) {
          if (!mbar_wait(smem_u32(&full[stage]), ph, abort_flag, a.err)) { ok = false; break; }
          fence_proxy_async();
          tc_fence_after();
          const uint32_t sa = smem_u32(stages + stage * stage_bytes);
          const uint32_t sb = sa + T::NPL * a_plane;
#pragma unroll
          for (int j = 0; j < TC_KP * T::ESZ / 32; ++j) {
            const uint32_t koff = (uint32_t)j * 256u;
            const uint32_t first = (kc > 0 || j > 0) ? 1u : 0u;
            const uint64_t ad = smem_desc(sa + koff, 128, sbo);
            const uint64_t bd = smem_desc(sb + koff, 128, sbo);
            tc_mma<MODE>(d_tmem, ad, bd, idesc, first);
            if constexpr (MODE == TC_BF16X3) {
              const uint64_t bdl = smem_desc(sb + b_plane + koff, 128, sbo);
              const uint64_t adl = smem_desc(sa + a_plane + koff, 128, sbo);
              tc_mma<MODE>(d_tmem, ad, bdl, idesc, 1u);
              tc_mma<MODE>(d_tmem, adl, bd, idesc, 1u);
            }
          }
          tc_commit(smem_u32(&empty[stage]));
          if (++stage == TC_STAGES) {
            stage = 0;
            ph ^= 1;
          }
        }
        if (!ok) break;
        tc_commit(smem_u32(&tfull[acc]));
      }
      // drain: every MMA issued so far completes before the CTA frees TMEM
      tc_commit(smem_u32(fin));
      mbar_wait(smem_u32(fin), 0, abort_flag, a.err);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- epilogue
    const int row = warp * 32 + lane;
    int64_t it = 0;
    for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++it) {
      const int acc = (int)(it & 1);
      const uint32_t aph = (uint32_t)((it >> 1) & 1);
      if (!mbar_wait(smem_u32(&tfull[acc]), aph, abort_flag, a.err)) break;
      tc_fence_after();
      const int nt = (int)(tile % a.n_nt);
      const int64_t rest = tile / a.n_nt;
      const int mt = (int)(rest % a.n_mt);
      const int inst = (int)(rest / a.n_mt);
      float2* C = g.C + inst_offset(inst, g.c_istride, g.c_bpos, g.nb) +
                  deposit_hi((uint64_t)mt, g.c_mpos, g.tm, g.nm) +
                  deposit_hi((uint64_t)nt, g.c_npos, a.tnb, g.nn);
      const bool row_ok = row < tmv;
      const int64_t crow = offCm[row];
      for (int c0 = 0; c0 < ncp; c0 += 32) {
        float v[32];
        tmem_ld32(tmem_base + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * ncp + c0), v);
        if (row_ok) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = c0 / 2 + j;
            if (n < tnv) C[crow + offCn[n]] = make_float2(v[2 * j], v[2 * j + 1]);
          }
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&tempty[acc]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == TC_MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TC_TMEM_COLS)
                 : "memory");
  }
}

}  // namespace tnx
