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
// Precision modes: TF32 (kind::tf32, one MMA per K step), BF16X3 (kind::f16
// with bf16 hi/lo split operands: hi*hi + hi*lo + lo*hi, FP32 accumulation in
// TMEM) and FP16X3 (the same with fp16 halves, each operand first scaled by a
// power of two from its largest component; the epilogue undoes it exactly).
// CM = 3 forms three real products instead (3M: T1 = Ar Br, T2 = Ai Bi,
// T3 = (Ar + Ai)(Br + Bi) in three accumulators; Re = T1 - T2,
// Im = T3 - T1 - T2), see TcPl.
//
// A (the large, streamed operand) is gathered by loader warps straight from
// its tensor's storage order -- the index permutation of Eq. (2) is folded into
// the loads, as in the paper's fused permutation-multiplication (SI, figure
// S7a).  B' (small) is written once per step by k_tc_prep_b in the exact
// shared-memory image of every (n tile, k chunk) and fetched by one bulk copy.
//
// Roles (480 threads, one CTA per SM, persistent over tiles):
//   warps 0-3  epilogue: TMEM -> registers -> C (lane = tile row)
//   warp  4    TMEM allocation; lane 0 issues tcgen05.mma and commits
//              (on an SM pair: lane 0 of the even CTA; the odd CTA's lane 0
//              forwards its readiness to the even CTA's barriers)
//   warps 5-12 loaders: A gathers into the A ring, or, when A is fetched by
//              TMA (and is not the TF32 4M operand itself), the fp32 ->
//              operand-plane converters (in place)
//   warp  13   A producer: when A is stored as [contracted..., free...] its
//              tiles are fetched by one tensor-map load per k chunk
//   warp  14   B' producer: one bulk copy of the (n tile, k chunk) image per k
//              chunk (two, of half planes, on an SM pair)
// Two rings decouple the operands: a deep ring of 16-32 KB A slots (more of
// the streamed operand in flight for the memory-bound steps) and a shallower
// ring of B' slots (B' comes from L2); a chunk's A and B' complete on the A
// slot's barrier, so the MMA thread waits once per chunk.
// SM pairs (PAIR): 2-CTA clusters, the even CTA issuing cta_group::2 MMAs of
// 256 rows over both CTAs' shared memory and TMEM.
// Every mbarrier wait is bounded by a globaltimer deadline; on expiry the
// kernel records TN_ERR_TIMEOUT in *err, every role leaves its loop, and the
// CTA frees its TMEM and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels_common.cuh"

namespace tnx {

constexpr int TC_M = 128;
constexpr int TC_TK = 16;            // complex k per pipeline stage
constexpr int TC_KP = 2 * TC_TK;     // real K' per stage
constexpr int TC_MAX_A = 8;           // A ring slots
constexpr int TC_MAX_B = 8;           // B' ring slots
constexpr int TC_MAX_ACC = 8;         // TMEM accumulator sets
constexpr int TC_EPI_WARPS = 4;
constexpr int TC_MMA_WARP = 4;
constexpr int TC_LOAD_WARPS = 8;
constexpr int TC_LOAD_THREADS = TC_LOAD_WARPS * 32;
constexpr int TC_PROD_WARP = TC_EPI_WARPS + 1 + TC_LOAD_WARPS;   // A producer (TMA)
constexpr int TC_B_WARP = TC_PROD_WARP + 1;                        // B' producer
constexpr int TC_THREADS = (TC_B_WARP + 1) * 32;
// one A slot: the fp32 tile of a k chunk (128 rows x 32 real), which is also
// the size of its TF32 plane and of its two BF16 planes
constexpr int TC_A_SLOT = TC_M * TC_KP * 4;
constexpr int TC_TMEM_COLS = 512;
constexpr uint64_t TC_WAIT_NS = 4000000000ull;           // 4 s per wait
constexpr int TC_MIN_SMEM = 120 * 1024;                  // keeps one CTA per SM
constexpr int TC_MAX_SMEM = 227 * 1024;                  // the dynamic shared-memory opt-in

enum TcMode { TC_TF32 = 0, TC_BF16X3 = 1, TC_FP16X3 = 2 };

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
template <>
struct TcT<TC_FP16X3> {   // operands scaled by powers of two into the FP16 range
  static constexpr int ESZ = 2, NPL = 2, FMT = 0;
};

// bytes of one operand plane per stage: rows x 32 real elements
__host__ __device__ constexpr int tc_plane_bytes(int rows, int esz) { return rows * TC_KP * esz; }
// Each plane row holds the stage's 32 real K' elements: 128 bytes for TF32,
// 64 bytes for BF16.  Planes use the tensor cores' K-major swizzled layouts
// (128-byte swizzle for 128-byte rows, 64-byte swizzle for 64-byte rows): row r
// of an 8-row group sits at r * rowbytes and its 16-byte chunk c at chunk
// position c ^ s(r), s(r) = r % 8 (128B) or (r / 2) % 4 (64B).  Writes of one
// chunk by 8 consecutive rows, and of all chunks of one row, are both free of
// bank conflicts.
__host__ __device__ constexpr int tc_rowbytes(int esz) { return TC_KP * esz; }
__host__ __device__ constexpr int tc_sbo(int esz) { return 8 * tc_rowbytes(esz); }
__host__ __device__ inline int tc_elem_off(int row, int kp, int esz) {
  const int byte = kp * esz;
  const int c = byte >> 4;
  const int sw = esz == 4 ? (row & 7) : ((row >> 1) & 3);
  return (row >> 3) * tc_sbo(esz) + (row & 7) * tc_rowbytes(esz) + ((c ^ sw) << 4) + (byte & 15);
}

// Operand planes of one k chunk (16 complex k) for 4M or 3M products.
//   4M: A' rows are the interleaved (re, im) storage itself, 32 real K'
//       (TF32: one plane; BF16: hi and lo planes); B' holds the 2x2 real form
//       of each B entry, two plane rows per complex column.
//   3M (T1 = Ar Br, T2 = Ai Bi, T3 = (Ar + Ai)(Br + Bi); Re = T1 - T2,
//       Im = T3 - T1 - T2): TF32 planes [Ar | Ai] and [As | unused]; BF16
//       planes [Ar_hi | Ai_hi], [Ar_lo | Ai_lo], [As_hi | As_lo]; B likewise
//       with Br, Bi, Bs, one plane row per complex column.  Sums are formed in
//       FP32 before rounding or splitting.
template <int MODE, int CM>
struct TcPl {
  static constexpr int ESZ = TcT<MODE>::ESZ;
  static constexpr int PLANES = CM == 4 ? TcT<MODE>::NPL : (MODE == TC_TF32 ? 2 : 3);
  static constexpr int ROWS_PER_COL = CM == 4 ? 2 : 1;   // B plane rows per complex column
  static constexpr int ACC_PER_COL = CM == 4 ? 2 : 3;    // TMEM columns per complex column
  static constexpr int A_PLANE = TC_M * TC_KP * ESZ;
  static constexpr int RAW = TC_M * TC_KP * 4;             // the fp32 tile a TMA load brings
  static constexpr int A_SLOT = PLANES * A_PLANE > RAW ? PLANES * A_PLANE : RAW;
  static constexpr int MIN_TN_C = CM == 4 ? 8 : 16;       // keeps the MMA's N a multiple of 16
};

struct TcArgs {
  GemmArgs g;
  const uint8_t* bimg;   // B' images, [inst][n tile][k chunk] blocks
  int32_t tn_c;          // complex columns per tile (>= 8); N' = 2 tn_c
  int32_t tnb;           // n bits covered by a tile (valid columns = 2^tnb)
  int32_t n_mt, n_nt, n_kc;
  int64_t n_tiles;
  int32_t* err;
  int32_t a_tma;         // 1: A tiles by tensor-map loads (A stored as [k..., m...])
  int32_t a_box_bytes;   // bytes one A tensor-map load brings: 2^tm rows x 128 bytes
  int32_t na;            // A ring slots (TcPl::A_SLOT bytes each)
  int32_t nbs;           // B' ring slots (one (n tile, k chunk) image each)
  int32_t fa_count;      // arrivals expected on an A slot's "full" barrier
  int32_t n_acc;         // TMEM accumulator sets (1..8), as many as fit 512 columns: the MMAs
                         // run up to n_acc tiles ahead of the epilogue (3M 128-column tiles: 1)
  int32_t nmw;           // m bits that are tensor-map rows (contiguous after the k bits)
  int32_t hi_shift;      // storage position where tensor-map dimension 2 starts
  int64_t c2_inst_mul;   // dimension-2 step per linear instance (tn_contract_pair batches)
  // epilogue write-back order: the 9 bits of a warp's 32-row x 16-column output
  // block sorted by their storage position in C (sel = index | 64 for columns)
  int32_t epi_ok;
  int8_t epi_sel[9], epi_pos[9];
  // split-K: tile t covers k chunks [s*kc_per, (s+1)*kc_per) with s = t % n_split
  // of output tile t / n_split; with n_split > 1 each split writes its partial C
  // (in C's layout) at c_part + s * c_part_stride and k_split_reduce adds them
  int32_t n_split;
  float2* c_part;
  int64_t c_part_stride;
  int32_t ls_split, ls_nt, ls_mt, ls_kc;   // log2 of n_split, n_nt, n_mt, n_kc (powers of two)
  // SM pairs: a work unit is a pair of m tiles (n_mt counts pairs); the CTA of
  // cluster rank r takes m tile 2 mt + r and the B' rows [r N'/2, (r + 1) N'/2)
  int32_t pair;
  // 1: each CTA (pair) runs all n tiles of one A block back to back (the block's
  // later reads come from L2 right after the first); 0: work units in index order
  int32_t nt_inner;
};

// Work unit `tile` -> split index, n tile, m tile, instance: shifts and masks
// (the extents are powers of two), cheap enough for one-chunk tiles.
struct TileIdx {
  int s, nt, mt, inst;
};
__device__ __forceinline__ TileIdx tile_decode(int64_t tile, const TcArgs& a) {
  TileIdx r;
  r.s = (int)(tile & (int64_t)(a.n_split - 1));
  const int64_t otile = tile >> a.ls_split;
  r.nt = (int)(otile & (int64_t)(a.n_nt - 1));
  const int64_t rest = otile >> a.ls_nt;
  r.mt = (int)(rest & (int64_t)(a.n_mt - 1));
  r.inst = (int)(rest >> a.ls_mt);
  return r;
}
constexpr int TC_EPI_STRIDE = 17;                                  // staging row stride (float2)
constexpr int TC_EPI_BYTES = TC_EPI_WARPS * 32 * TC_EPI_STRIDE * 8;  // epilogue staging

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
// DRAIN: keep waiting after an abort (for work already in flight), still
// within the limit.
template <bool DRAIN = false>
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag, int32_t* err,
                                          uint64_t limit_ns = TC_WAIT_NS) {
  if (mbar_try_wait(a, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(a, parity)) return true;
    if ((i & 255) == 0) {
      if (!DRAIN && *abort_flag) return false;
      if (gtimer() - t0 > limit_ns) {
        *abort_flag = 1;
        atomicExch(err, TN_ERR_TIMEOUT);
        return false;
      }
    }
  }
}
// Self-test of the bounded wait: one thread waits on an mbarrier that nothing
// ever arrives on; the wait must give up after limit_ns and record the timeout.
__global__ void k_selftest_wait(int32_t* err, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool ok = mbar_wait(smem_u32(&bar), 0, &abort_flag, err, limit_ns);
    if (ok) atomicExch(err, 1);
  }
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(a),
               "r"(bytes)
               : "memory");
}
// Barrier over `nthreads` threads (named barrier `id`) that also returns the
// OR of `pred` over them, so that all of them take the same branch after it.
__device__ __forceinline__ bool named_barrier_or(int id, int nthreads, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
      : "memory");
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
// ---- SM pairs (cta_group::2): two CTAs of a 2-CTA cluster share each MMA
// (M = 256: 128 A rows and half of B' in each CTA's shared memory, each CTA's
// accumulator rows in its own TMEM); the even CTA issues the MMAs.
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// shared::cluster address of the object at CTA-local shared address `a` in CTA `rank`
__device__ __forceinline__ uint32_t mapa_cta(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// One arrival on a barrier of the peer CTA.  The default (CTA-scope) release:
// the cluster-scope form waits for every outstanding memory operation first
// (measured ~1,700 cycles per arrival under the epilogue's store stream), and
// what it would order here -- operand writes to this CTA's own shared memory,
// completed before the local barrier the caller waited on -- needs no more.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// commit of the pair's MMAs: one arrival on the barrier at this offset in both CTAs
__device__ __forceinline__ void tc_commit_pair(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          mbar),
      "h"((uint16_t)3)
      : "memory");
}
template <bool PAIR>
__device__ __forceinline__ void tc_commit_g(uint32_t mbar) {
  if constexpr (PAIR)
    tc_commit_pair(mbar);
  else
    tc_commit(mbar);
}
// every thread of both CTAs of the cluster
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared-memory matrix descriptor, K-major swizzled: start address, leading
// byte offset (unused for swizzled K-major, encoded as 16 B), stride byte
// offset between 8-row groups, descriptor version 1, layout type (2 = 128-byte
// swizzle, 4 = 64-byte swizzle)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo, uint32_t layout) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)layout << 61;
  return d;
}
// One MMA; the operand descriptors are given as their low words (start
// address) and the high word they share (stride, version, layout).
template <int MODE, bool PAIR = false>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint32_t adesc_lo, uint32_t bdesc_lo, uint32_t desc_hi,
                                       uint32_t idesc, uint32_t accumulate) {
#define TC_MMA_ASM(GROUP, KIND)                                                                                   \
  asm volatile("{\n\t.reg .pred p;\n\t.reg .b64 ad, bd;\n\tmov.b64 ad, {%1, %3};\n\tmov.b64 bd, {%2, %3};\n\t"    \
               "setp.ne.b32 p, %5, 0;\n\t"                                                                         \
               "tcgen05.mma.cta_group::" GROUP ".kind::" KIND " [%0], ad, bd, %4, p;\n\t}" ::"r"(d_tmem),           \
               "r"(adesc_lo), "r"(bdesc_lo), "r"(desc_hi), "r"(idesc), "r"(accumulate)                            \
               : "memory")
  if constexpr (MODE == TC_TF32) {
    if constexpr (PAIR)
      TC_MMA_ASM("2", "tf32");
    else
      TC_MMA_ASM("1", "tf32");
  } else {
    if constexpr (PAIR)
      TC_MMA_ASM("2", "f16");
    else
      TC_MMA_ASM("1", "f16");
  }
#undef TC_MMA_ASM
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

// Three 16-column TMEM loads (the 3M accumulators T1, T2, T3 of one 16-column
// block) and the wait for them, in one asm statement so that no register is
// read before the wait.
__device__ __forceinline__ void tmem_ld16x3(uint32_t t1, uint32_t t2, uint32_t t3, float* v) {
  uint32_t r[48];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%48];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%49];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47}, [%50];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47])
      : "r"(t1), "r"(t2), "r"(t3)
      : "memory");
#pragma unroll
  for (int i = 0; i < 48; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t w;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(w) : "f"(x));
  return w;
}
// hi = round(x), lo = round(x - hi) in the 16-bit operand type, for a pair of
// consecutive K elements (packed low element first)
template <int MODE>
__device__ __forceinline__ void split_pair(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  if constexpr (MODE == TC_FP16X3) {
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  }
}
// the operand scale of a mode: 2^s from the tensor's recorded maximum (FP16X3), else 1
template <int MODE>
__device__ __forceinline__ float operand_scale(const float* amax) {
  if constexpr (MODE == TC_FP16X3)
    return pow2f(fp16_scale_exp(amax));
  else
    return 1.f;
}
__device__ __forceinline__ void st16(uint8_t* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  *reinterpret_cast<uint4*>(p) = make_uint4(a, b, c, d);
}
// 3M A planes for 8 consecutive complex k (k = 8h .. 8h+7 of the chunk) of tile
// row `row`, from their values x[i] = (re, im)
template <int MODE>
__device__ __forceinline__ void put3m(uint8_t* sa, int row, int h, const float2 (&x)[8], float sc) {
  constexpr int AP = TcPl<MODE, 3>::A_PLANE;
  if constexpr (MODE == TC_TF32) {
    uint32_t r[8], i[8], s[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      r[e] = to_tf32(x[e].x);
      i[e] = to_tf32(x[e].y);
      s[e] = to_tf32(x[e].x + x[e].y);
    }
    st16(sa + tc_elem_off(row, 8 * h, 4), r[0], r[1], r[2], r[3]);
    st16(sa + tc_elem_off(row, 8 * h + 4, 4), r[4], r[5], r[6], r[7]);
    st16(sa + tc_elem_off(row, 16 + 8 * h, 4), i[0], i[1], i[2], i[3]);
    st16(sa + tc_elem_off(row, 16 + 8 * h + 4, 4), i[4], i[5], i[6], i[7]);
    st16(sa + AP + tc_elem_off(row, 8 * h, 4), s[0], s[1], s[2], s[3]);
    st16(sa + AP + tc_elem_off(row, 8 * h + 4, 4), s[4], s[5], s[6], s[7]);
  } else {
    uint32_t rh[4], rl[4], ih[4], il[4], sh[4], sl[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 u = x[2 * q], w = x[2 * q + 1];
      split_pair<MODE>(u.x * sc, w.x * sc, rh[q], rl[q]);
      split_pair<MODE>(u.y * sc, w.y * sc, ih[q], il[q]);
      split_pair<MODE>((u.x + u.y) * sc, (w.x + w.y) * sc, sh[q], sl[q]);
    }
    st16(sa + tc_elem_off(row, 8 * h, 2), rh[0], rh[1], rh[2], rh[3]);
    st16(sa + tc_elem_off(row, 16 + 8 * h, 2), ih[0], ih[1], ih[2], ih[3]);
    st16(sa + AP + tc_elem_off(row, 8 * h, 2), rl[0], rl[1], rl[2], rl[3]);
    st16(sa + AP + tc_elem_off(row, 16 + 8 * h, 2), il[0], il[1], il[2], il[3]);
    st16(sa + 2 * AP + tc_elem_off(row, 8 * h, 2), sh[0], sh[1], sh[2], sh[3]);
    st16(sa + 2 * AP + tc_elem_off(row, 16 + 8 * h, 2), sl[0], sl[1], sl[2], sl[3]);
  }
}

// ------------------------------------------------------------------ B' images
// One thread per 16-byte chunk of every (instance, n tile, k chunk) block:
// reads the complex B entries the chunk covers and writes their 2x2 real form
// (split into hi/lo planes for BF16X3) in the block's shared-memory image.
// Threads run in memory order of the image, so the writes are contiguous.
// Padding (k or n beyond the operand) is zero.
template <int MODE>
__global__ void __launch_bounds__(256) k_tc_prep_b(const TcArgs a) {
  using T = TcT<MODE>;
  constexpr int KPC = 16 / (2 * T::ESZ);        // complex k per 16-byte chunk (2 or 4)
  constexpr int CPR = TC_KP * T::ESZ / 16;      // chunks per row (8 or 4)
  const GemmArgs& g = a.g;
  const int ncp = 2 * a.tn_c;
  const int plane = tc_plane_bytes(ncp, T::ESZ);
  const int64_t block_bytes = (int64_t)T::NPL * plane;
  const int per_block = ncp * CPR;              // chunks per plane
  const int tkv = 1 << g.tk, tnv = 1 << a.tnb;
  const float sc = operand_scale<MODE>(g.amax_b);
  // offsets in B of the k inside a chunk and of the n inside a tile (-1: padding)
  __shared__ int64_t koff[TC_TK];
  __shared__ int64_t noff[128];
  for (int i = threadIdx.x; i < TC_TK; i += blockDim.x) koff[i] = i < tkv ? deposit_hi((uint64_t)i, g.b_kpos, 0, g.tk) : -1;
  for (int i = threadIdx.x; i < 128; i += blockDim.x) noff[i] = i < tnv ? deposit_hi((uint64_t)i, g.b_npos, 0, a.tnb) : -1;
  __syncthreads();
  const int64_t n_blocks = (int64_t)g.n_inst << (a.ls_nt + a.ls_kc);
  // one CTA per (instance, n tile, k chunk) block at a time; threads walk the
  // block's 16-byte chunks in memory order of the image
  for (int64_t blk = blockIdx.x; blk < n_blocks; blk += gridDim.x) {
    const int kc = (int)(blk & (a.n_kc - 1));
    const int nt = (int)((blk >> a.ls_kc) & (a.n_nt - 1));
    const int inst = (int)(blk >> (a.ls_kc + a.ls_nt));
    const int64_t base = inst_offset(inst, g.b_istride, g.b_bpos, g.nb) + deposit_hi((uint64_t)kc, g.b_kpos, g.tk, g.nk) +
                         deposit_hi((uint64_t)nt, g.b_npos, a.tnb, g.nn);
    uint8_t* dblk = const_cast<uint8_t*>(a.bimg) + blk * block_bytes;
    for (int q = threadIdx.x; q < per_block; q += blockDim.x) {
      // q in image order: row within the 8-row group fastest, then chunk, then group
      const int rlo = q & 7, c = (q >> 3) % CPR, rg = (q >> 3) / CPR;
      const int row = rg * 8 + rlo;
      const int t = row & 1, nl = row >> 1;
      const int64_t no = noff[nl];
      float vals[2 * KPC];
#pragma unroll
      for (int i = 0; i < KPC; ++i) {
        const int64_t ko = koff[c * KPC + i];
        float2 b = make_float2(0.f, 0.f);
        if (no >= 0 && ko >= 0) b = g.B[base + no + ko];
        // row (n, t), columns (k, u): t = 0 -> (Re, -Im), t = 1 -> (Im, Re)
        vals[2 * i] = t ? b.y : b.x;
        vals[2 * i + 1] = t ? b.x : -b.y;
      }
      uint8_t* dst = dblk + tc_elem_off(row, c * KPC * 2, T::ESZ);
      if constexpr (MODE == TC_TF32) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = to_tf32(vals[i]);
        *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
      } else {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) split_pair<MODE>(vals[2 * i] * sc, vals[2 * i + 1] * sc, hi[i], lo[i]);
        *reinterpret_cast<uint4*>(dst) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(dst + plane) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
    }
  }
}

// 3M B images: per (instance, n tile, k chunk) block the planes of TcPl<MODE, 3>,
// one plane row per complex column n; one thread per 16-byte chunk in memory
// order of the image.  Padding (k or n beyond the operand) is zero.
template <int MODE>
__global__ void __launch_bounds__(256) k_tc_prep_b3(const TcArgs a) {
  using P = TcPl<MODE, 3>;
  constexpr int ESZ = P::ESZ;
  constexpr int EPC = 16 / ESZ;                 // elements per 16-byte chunk (4 or 8)
  constexpr int CPR = TC_KP * ESZ / 16;         // chunks per plane row (8 or 4)
  const GemmArgs& g = a.g;
  const int rows = a.tn_c;
  const int plane = tc_plane_bytes(rows, ESZ);
  const int64_t block_bytes = (int64_t)P::PLANES * plane;
  const int per_block = P::PLANES * rows * CPR;
  const int per_plane = rows * CPR;
  const int tkv = 1 << g.tk, tnv = 1 << a.tnb;
  const float sc = operand_scale<MODE>(g.amax_b);
  __shared__ int64_t koff[TC_TK];
  __shared__ int64_t noff[128];
  for (int i = threadIdx.x; i < TC_TK; i += blockDim.x) koff[i] = i < tkv ? deposit_hi((uint64_t)i, g.b_kpos, 0, g.tk) : -1;
  for (int i = threadIdx.x; i < 128; i += blockDim.x) noff[i] = i < tnv ? deposit_hi((uint64_t)i, g.b_npos, 0, a.tnb) : -1;
  __syncthreads();
  const int64_t n_blocks = (int64_t)g.n_inst << (a.ls_nt + a.ls_kc);
  for (int64_t blk = blockIdx.x; blk < n_blocks; blk += gridDim.x) {
    const int kc = (int)(blk & (a.n_kc - 1));
    const int nt = (int)((blk >> a.ls_kc) & (a.n_nt - 1));
    const int inst = (int)(blk >> (a.ls_kc + a.ls_nt));
    const int64_t base = inst_offset(inst, g.b_istride, g.b_bpos, g.nb) + deposit_hi((uint64_t)kc, g.b_kpos, g.tk, g.nk) +
                         deposit_hi((uint64_t)nt, g.b_npos, a.tnb, g.nn);
    uint8_t* dblk = const_cast<uint8_t*>(a.bimg) + blk * block_bytes;
    for (int pq = threadIdx.x; pq < per_block; pq += blockDim.x) {
      const int pl = pq / per_plane, q = pq % per_plane;
      const int rlo = q & 7, c = (q >> 3) % CPR, rg = (q >> 3) / CPR;
      const int n = rg * 8 + rlo;
      const int half = c / (CPR / 2), k0 = (c % (CPR / 2)) * EPC;   // k0.. within the half's 16 k
      const int64_t no = noff[n];   // n < tn_c <= 128
      float2 b[8];
#pragma unroll
      for (int i = 0; i < EPC; ++i) {
        const int64_t ko = koff[k0 + i];
        b[i] = (no >= 0 && ko >= 0) ? g.B[base + no + ko] : make_float2(0.f, 0.f);
      }
      uint8_t* dst = dblk + (int64_t)pl * plane + tc_elem_off(n, c * EPC, ESZ);
      if constexpr (MODE == TC_TF32) {
        // plane 0: [Br | Bi]; plane 1: [Bs | 0]
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float v = pl == 0 ? (half == 0 ? b[i].x : b[i].y) : (half == 0 ? b[i].x + b[i].y : 0.f);
          w[i] = to_tf32(v);
        }
        st16(dst, w[0], w[1], w[2], w[3]);
      } else {
        // plane 0: [Br_hi | Bi_hi]; plane 1: [Br_lo | Bi_lo]; plane 2: [Bs_hi | Bs_lo]
        uint32_t w[4];
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) {
          const float2 u = b[2 * q2], v = b[2 * q2 + 1];
          float x0, x1;
          if (pl < 2) {
            x0 = half == 0 ? u.x : u.y;
            x1 = half == 0 ? v.x : v.y;
          } else {
            x0 = u.x + u.y;
            x1 = v.x + v.y;
          }
          uint32_t hi, lo;
          split_pair<MODE>(x0 * sc, x1 * sc, hi, lo);
          w[q2] = (pl == 0 || (pl == 2 && half == 0)) ? hi : lo;
        }
        st16(dst, w[0], w[1], w[2], w[3]);
      }
    }
  }
}

// Split-K: C[i] = sum over splits of the partials, in split order.
__global__ void k_split_reduce(const float2* __restrict__ part, int n_split, int64_t stride,
                               float2* __restrict__ C, int64_t n, float* amax_c) {
  float am = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float2 acc = part[i];
    for (int sp = 1; sp < n_split; ++sp) {
      const float2 v = part[sp * stride + i];
      acc.x += v.x;
      acc.y += v.y;
    }
    C[i] = acc;
    am = fmaxf(am, cabs_max(acc));
  }
  if (amax_c) amax_update(amax_c, am);   // blockDim is a multiple of 32
}

// ------------------------------------------------------------------ the GEMM
template <int MODE, int CM, bool PAIR>
__global__ void __launch_bounds__(TC_THREADS, 1) k_cgemm_tc(const __grid_constant__ TcArgs a,
                                                              const __grid_constant__ CUtensorMap tma_a) {
  using T = TcT<MODE>;
  using P = TcPl<MODE, CM>;
  static_assert(!PAIR || CM == 4, "SM pairs form 4M products");
  extern __shared__ __align__(1024) uint8_t smem_dyn[];
  // swizzle atoms need 1024-byte aligned slots
  uint8_t* smem_raw = smem_dyn + ((1024 - (smem_u32(smem_dyn) & 1023)) & 1023);
  const GemmArgs& g = a.g;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncp = 2 * a.tn_c;                                   // real columns of C per tile
  const int setw = P::ACC_PER_COL * a.tn_c;                     // TMEM columns per accumulator set
  const int a_plane = P::A_PLANE;
  // B' planes: the image's (all N' rows) and this CTA's (half of them for a pair)
  const int b_plane_g = tc_plane_bytes(P::ROWS_PER_COL * a.tn_c, T::ESZ);
  const int b_plane = PAIR ? b_plane_g / 2 : b_plane_g;
  // the pair's rank, and the work units of this CTA (pairs take them together)
  const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
  const int64_t t_first = PAIR ? (int64_t)(blockIdx.x >> 1) : (int64_t)blockIdx.x;
  const int64_t t_step = PAIR ? (int64_t)(gridDim.x >> 1) : (int64_t)gridDim.x;
  auto own_mt = [&](int mt) { return PAIR ? 2 * mt + (int)rank : mt; };
  // the j-th work unit of this CTA (pair), -1 past the last: units t_first,
  // t_first + t_step, ... in index order, or -- nt_inner -- groups (split index,
  // m tile, instance) taken that way with all their n tiles in turn
  const int64_t n_groups = a.n_tiles >> a.ls_nt;
  auto seq_tile = [&](int64_t j) -> int64_t {
    if (!a.nt_inner) {
      const int64_t t = t_first + j * t_step;
      return t < a.n_tiles ? t : -1;
    }
    const int64_t gi = t_first + (j >> a.ls_nt) * t_step;
    if (gi >= n_groups) return -1;
    const int64_t sp = gi & (int64_t)(a.n_split - 1), rest = gi >> a.ls_split;
    return sp | ((j & (int64_t)(a.n_nt - 1)) << a.ls_split) | (rest << (a.ls_split + a.ls_nt));
  };
  // FP16X3: A and B enter scaled by 2^sa, 2^sb; the epilogue multiplies by 2^-sa 2^-sb (exact)
  const float sc_a = operand_scale<MODE>(g.amax_a);
  const float us_a = 1.f / sc_a, us_b = 1.f / operand_scale<MODE>(g.amax_b);
  const int b_slot = P::PLANES * b_plane;
  const int64_t b_slot_g = (int64_t)P::PLANES * b_plane_g;
  const int na = a.na, nbs = a.nbs;
  uint8_t* aring = smem_raw;
  uint8_t* bring = aring + na * P::A_SLOT;
  uint64_t* bars = reinterpret_cast<uint64_t*>(bring + nbs * b_slot);
  uint64_t* fullA = bars;
  uint64_t* emptyA = bars + TC_MAX_A;
  uint64_t* rawA = bars + 2 * TC_MAX_A;
  // (a chunk's B' copy also completes on fullA of the chunk's A slot, and B'
  // slots are released through emptyA: the B' ring has no barriers of its own)
  uint64_t* tfull = bars + 3 * TC_MAX_A;
  uint64_t* tempty = tfull + TC_MAX_ACC;
  uint64_t* fin = tempty + TC_MAX_ACC;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int64_t* offCm = reinterpret_cast<int64_t*>(tmem_slot + 4);
  float2* epi_stage = reinterpret_cast<float2*>(reinterpret_cast<uint8_t*>(bars) + 4096);
  int64_t* offCn = offCm + TC_M;

  // zero every slot once: padding rows / columns are never written again
  for (int i = threadIdx.x; i < (na * P::A_SLOT + nbs * b_slot) / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(aring)[i] = make_uint4(0, 0, 0, 0);
  const int tmv = 1 << g.tm, tnv = 1 << a.tnb;
  for (int r = threadIdx.x; r < TC_M; r += blockDim.x)
    offCm[r] = r < tmv ? deposit_hi((uint64_t)r, g.c_mpos, 0, g.tm) : 0;
  for (int c = threadIdx.x; c < 128; c += blockDim.x)
    offCn[c] = c < tnv ? deposit_hi((uint64_t)c, g.c_npos, 0, a.tnb) : 0;
  if (threadIdx.x == 0) {
    // SM pairs: the even CTA's fullA and tempty also take one arrival from the
    // odd CTA per phase (its chunk in place, its accumulator set drained)
    const uint32_t peer = (PAIR && rank == 0) ? 1u : 0u;
    for (int s = 0; s < na; ++s) {
      mbar_init(smem_u32(&fullA[s]), a.fa_count + 1 + peer);   // + the B' producer's arrival
      mbar_init(smem_u32(&emptyA[s]), 1);
      mbar_init(smem_u32(&rawA[s]), 1);
    }
    for (int i = 0; i < TC_MAX_ACC; ++i) {
      mbar_init(smem_u32(&tfull[i]), 1);
      mbar_init(smem_u32(&tempty[i]), TC_EPI_WARPS * 32 + peer);
    }
    mbar_init(smem_u32(fin), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == TC_MMA_WARP) {
    // a pair allocates together: one warp in each of its two CTAs, unconditionally
    if constexpr (PAIR) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(TC_TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(TC_TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  // a pair's barriers are initialised and its TMEM allocated in both CTAs
  // before either CTA's arrivals or MMAs reach the other
  if constexpr (PAIR) cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int kc_n = a.n_kc;
  const int kc_per = a.n_kc / a.n_split;

  if (warp == TC_PROD_WARP) {
    // ---------------------------------------------------------------- A producer (TMA)
    if (a.a_tma && lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tma_a)) : "memory");
      int slot = 0;
      uint32_t ph = 0;
      bool ok = true;
      int64_t issued = 0;
      int64_t jt = 0;
      for (int64_t tile = seq_tile(0); tile >= 0 && ok; tile = seq_tile(++jt)) {
        const TileIdx ti = tile_decode(tile, a);
        const int kc0 = ti.s * kc_per;
        const int mt = own_mt(ti.mt), inst = ti.inst;
        // tensor-map coordinates of the tile: rows from the m bits after the
        // first tm, dimension 2 from the remaining m bits and the instance bits
        const int c1 = (mt & ((1 << (a.nmw - g.tm)) - 1)) << g.tm;
        int64_t c2 = (int64_t)inst * a.c2_inst_mul;
        for (int i = a.nmw; i < g.nm; ++i)
          if ((mt >> (i - g.tm)) & 1) c2 += (int64_t)1 << (g.a_mpos[i] - a.hi_shift);
        for (int j = 0; j < g.nb; ++j)
          if ((inst >> j) & 1) c2 += (int64_t)1 << (g.a_bpos[j] - a.hi_shift);
        for (int kc = kc0; kc < kc0 + kc_per; ++kc) {
          if (!mbar_wait(smem_u32(&emptyA[slot]), ph ^ 1, abort_flag, a.err)) { ok = false; break; }
          // TF32 4M: the tile is the MMA operand; otherwise converted in place first
          const uint32_t bar = (MODE == TC_TF32 && CM == 4) ? smem_u32(&fullA[slot]) : smem_u32(&rawA[slot]);
          mbar_arrive_expect_tx(bar, (uint32_t)a.a_box_bytes);
          tma_load_3d(smem_u32(aring + slot * P::A_SLOT), &tma_a, kc * TC_KP, c1, (int)c2, bar);
          ++issued;
          if (++slot == na) {
            slot = 0;
            ph ^= 1;
          }
        }
      }
      if (!ok) {
        // aborted: the loads still in flight (at most the last na) land before the CTA leaves
        uint64_t* txb = (MODE == TC_TF32 && CM == 4) ? fullA : rawA;
        for (int64_t j = issued - 1; j >= 0 && j >= issued - na; --j)
          mbar_wait<true>(smem_u32(&txb[j % na]), (uint32_t)((j / na) & 1), abort_flag, a.err,
                                 1000000000ull);
      }
    }
    __syncwarp();
  } else if (warp == TC_B_WARP) {
    // ---------------------------------------------------------------- B' producer
    if (lane == 0) {
      // B' slot q % nbs is free again once the MMAs of chunk q - nbs are done:
      // the MMA thread's single commit per chunk arrives on emptyA of that
      // chunk's A slot, whose completion for chunk j has parity (j / na) & 1
      // (na >= nbs, so that barrier cannot have moved on by a further phase).
      // The copy of chunk q completes on fullA of A slot q % na, whose previous
      // phase (chunk q - na <= q - nbs) the MMA thread has already passed, so
      // the MMA thread waits for A and B' of a chunk on one barrier.
      int slot = 0, ws = 0, sa = 0;
      uint32_t wph = 0;
      int64_t q = 0;
      bool ok = true;
      int64_t jt = 0;
      for (int64_t tile = seq_tile(0); tile >= 0 && ok; tile = seq_tile(++jt)) {
        const TileIdx ti = tile_decode(tile, a);
        const int kc0 = ti.s * kc_per;
        const int nt = ti.nt, inst = ti.inst;
        const uint8_t* bt = a.bimg + (((int64_t)inst * a.n_nt + nt) * kc_n) * b_slot_g;
        for (int kc = kc0; kc < kc0 + kc_per; ++kc, ++q) {
          if (q >= nbs) {
            if (!mbar_wait(smem_u32(&emptyA[ws]), wph, abort_flag, a.err)) { ok = false; break; }
            if (++ws == na) {
              ws = 0;
              wph ^= 1;
            }
          }
          const uint32_t fb = smem_u32(&fullA[sa]);
          mbar_arrive_expect_tx(fb, (uint32_t)b_slot);
          if constexpr (PAIR) {
            // this CTA's half of every plane: rows [rank N'/2, (rank + 1) N'/2)
#pragma unroll
            for (int pl = 0; pl < P::PLANES; ++pl)
              bulk_g2s(smem_u32(bring + slot * b_slot + pl * b_plane),
                       bt + (int64_t)kc * b_slot_g + pl * b_plane_g + (int)rank * b_plane, (uint32_t)b_plane, fb);
          } else {
            bulk_g2s(smem_u32(bring + slot * b_slot), bt + (int64_t)kc * b_slot, (uint32_t)b_slot, fb);
          }
          if (++slot == nbs) slot = 0;
          if (++sa == na) sa = 0;
        }
      }
      if (!ok) {
        // aborted: the copies still in flight (at most the last nbs) land before
        // the CTA leaves; their barriers also wait for A arrivals that an abort
        // may have cut off, so each wait is short (a copy lands in microseconds)
        for (int64_t j = q - 1; j >= 0 && j >= q - nbs; --j)
          mbar_wait<true>(smem_u32(&fullA[j % na]), (uint32_t)((j / na) & 1), abort_flag, a.err,
                          20000000ull);
      }
    }
    __syncwarp();
  } else if (warp >= TC_MMA_WARP + 1 && a.a_tma) {
    // ---------------------------------------------------------------- converters (TMA)
    // The fp32 tile (128 rows x 128 bytes, 128-byte swizzle) is read into
    // registers, then -- after a barrier of the group -- rewritten in place as
    // the operand planes: 4M BF16X3/FP16X3 hi and lo (128 rows x 64 bytes
    // each); 3M the planes of TcPl<MODE, 3> by items (row, 8 complex k).  The 8
    // warps form two groups of 4 that take alternate k chunks, so two chunks
    // are converted at once (the A ring has an even number of slots, so every
    // slot belongs to one group); rows past the tile's 2^tm are left alone.
    if constexpr (CM == 3 || MODE != TC_TF32) {
      const int lt = threadIdx.x - (TC_MMA_WARP + 1) * 32;
      constexpr int GT = TC_LOAD_THREADS / 2;                     // threads per group
      const int grp = lt / GT, glt = lt % GT;
      const int tmv = 1 << g.tm;
      // 4M: 512 items (row, 16-byte output chunk c); 3M: 256 items (row, half h)
      constexpr int NIT = CM == 3 ? 2 * TC_M / GT : TC_M * (TC_KP * T::ESZ / 16) / GT;
      int roff[NIT][4], woff[NIT], irow[NIT], isub[NIT];
#pragma unroll
      for (int j = 0; j < NIT; ++j) {
        const int q = glt + j * GT;
        irow[j] = q % TC_M;
        isub[j] = q / TC_M;
        if constexpr (CM == 3) {
#pragma unroll
          for (int r = 0; r < 4; ++r) roff[j][r] = tc_elem_off(irow[j], 16 * isub[j] + 4 * r, 4);
          woff[j] = 0;
        } else {
          roff[j][0] = tc_elem_off(irow[j], 8 * isub[j], 4);
          roff[j][1] = tc_elem_off(irow[j], 8 * isub[j] + 4, 4);
          roff[j][2] = roff[j][3] = 0;
          woff[j] = tc_elem_off(irow[j], 8 * isub[j], T::ESZ);
        }
      }
      int slot = 0;
      uint32_t ph = 0;
      int64_t chunk = 0;
      bool stop = false;
      int64_t jt = 0;
      for (int64_t tile = seq_tile(0); tile >= 0 && !stop; tile = seq_tile(++jt)) {
        for (int kc = 0; kc < kc_per; ++kc, ++chunk) {
          if ((int)(chunk & 1) == grp) {
            const bool got = mbar_wait(smem_u32(&rawA[slot]), ph, abort_flag, a.err);
            uint8_t* sa = aring + slot * P::A_SLOT;
            float4 x[NIT][CM == 3 ? 4 : 2];
#pragma unroll
            for (int j = 0; j < NIT; ++j)
              if (irow[j] < tmv) {
#pragma unroll
                for (int r = 0; r < (CM == 3 ? 4 : 2); ++r)
                  x[j][r] = *reinterpret_cast<const float4*>(sa + roff[j][r]);
              }
            // every thread of the group has read the tile; all agree whether to go on
            stop = named_barrier_or(1 + grp, GT, !got || *abort_flag);
            if (stop) break;
#pragma unroll
            for (int j = 0; j < NIT; ++j) {
              if (irow[j] >= tmv) continue;
              if constexpr (CM == 3) {
                float2 v[8];
#pragma unroll
                for (int r = 0; r < 4; ++r) {   // raw chunk 4h + r: complex k 8h + 2r, 8h + 2r + 1
                  v[2 * r] = make_float2(x[j][r].x, x[j][r].y);
                  v[2 * r + 1] = make_float2(x[j][r].z, x[j][r].w);
                }
                put3m<MODE>(sa, irow[j], isub[j], v, sc_a);
              } else {
                const float xs[8] = {x[j][0].x, x[j][0].y, x[j][0].z, x[j][0].w,
                                     x[j][1].x, x[j][1].y, x[j][1].z, x[j][1].w};
                uint32_t hi[4], lo[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) split_pair<MODE>(xs[2 * i] * sc_a, xs[2 * i + 1] * sc_a, hi[i], lo[i]);
                *reinterpret_cast<uint4*>(sa + woff[j]) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<uint4*>(sa + a_plane + woff[j]) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
              }
            }
            fence_proxy_async();
            mbar_arrive(smem_u32(&fullA[slot]));
          }
          if (++slot == na) {
            slot = 0;
            ph ^= 1;
          }
        }
      }
    }
  } else if (warp >= TC_MMA_WARP + 1) {
    // ---------------------------------------------------------------- loaders
    if constexpr (CM == 3) {
      // 3M: one item (tile row, 8 complex k) per thread, gathered from A's
      // storage order into registers; the next slot's item is in flight while
      // the current one is converted into the planes and stored
      const int lt = threadIdx.x - (TC_MMA_WARP + 1) * 32;
      const int row = lt % TC_M, h = lt / TC_M;
      const int tkv = 1 << g.tk;
      const bool rok = row < (1 << g.tm);
      const bool kadj = g.nk > 0 && g.a_kpos[0] == 0;
      int64_t goff[8];
      const int64_t roff = rok ? deposit_hi((uint64_t)row, g.a_mpos, 0, g.tm) : 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = 8 * h + i;
        goff[i] = (rok && k < tkv) ? roff + deposit_hi((uint64_t)k, g.a_kpos, 0, g.tk) : -1;
      }
      auto tile_base = [&](int64_t tile) -> const float2* {
        const TileIdx ti = tile_decode(tile, a);
        const int mt = own_mt(ti.mt), inst = ti.inst;
        return g.A + inst_offset(inst, g.a_istride, g.a_bpos, g.nb) +
               deposit_hi((uint64_t)mt, g.a_mpos, g.tm, g.nm);
      };
      auto issue = [&](float2(&v)[8], const float2* Ak) {
        const bool v16 = kadj && ((reinterpret_cast<uintptr_t>(Ak) & 15) == 0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t o0 = goff[2 * q], o1 = goff[2 * q + 1];
          if (v16 && o1 >= 0) {
            const float4 t = __ldg(reinterpret_cast<const float4*>(Ak + o0));
            v[2 * q] = make_float2(t.x, t.y);
            v[2 * q + 1] = make_float2(t.z, t.w);
          } else {
            v[2 * q] = o0 >= 0 ? __ldg(Ak + o0) : make_float2(0.f, 0.f);
            v[2 * q + 1] = o1 >= 0 ? __ldg(Ak + o1) : make_float2(0.f, 0.f);
          }
        }
      };
      int slot = 0;
      uint32_t ph = 0;
      int64_t jt = 0;
      int64_t tile = seq_tile(0);
      int kc = tile >= 0 ? (int)(tile & (int64_t)(a.n_split - 1)) * kc_per : 0;
      const float2* An = tile >= 0 ? tile_base(tile) : g.A;
      float2 v0[8], v1[8];
      auto body = [&](float2(&vc)[8], float2(&vn)[8]) -> bool {
        int64_t ntile = tile, njt = jt;
        int nkc = kc + 1;
        if (nkc == (int)(tile & (int64_t)(a.n_split - 1)) * kc_per + kc_per) {
          ntile = seq_tile(++njt);
          nkc = ntile >= 0 ? (int)(ntile & (int64_t)(a.n_split - 1)) * kc_per : 0;
          if (ntile >= 0) An = tile_base(ntile);
        }
        if (ntile >= 0) issue(vn, An + deposit_hi((uint64_t)nkc, g.a_kpos, g.tk, g.nk));
        uint8_t* sa = aring + slot * P::A_SLOT;
        if (!mbar_wait(smem_u32(&emptyA[slot]), ph ^ 1, abort_flag, a.err)) return false;
        if (rok) put3m<MODE>(sa, row, h, vc, sc_a);
        fence_proxy_async();
        mbar_arrive(smem_u32(&fullA[slot]));
        if (++slot == na) {
          slot = 0;
          ph ^= 1;
        }
        tile = ntile;
        jt = njt;
        kc = nkc;
        return true;
      };
      if (tile >= 0) issue(v0, An + deposit_hi((uint64_t)kc, g.a_kpos, g.tk, g.nk));
      while (tile >= 0) {
        if (!body(v0, v1) || tile < 0) break;
        if (!body(v1, v0)) break;
      }
    } else {
      // Thread lt owns tile row (lt % 128) and every other 16-byte chunk of it, so
      // the 32 lanes of a warp write 32 consecutive rows: four whole 8 x 16-byte
      // core matrices, free of bank conflicts whatever A's storage order.  A chunk
      // holds KPC consecutive complex k (2 for TF32, 4 for BF16); when the lowest
      // k bit is memory position 0 those are contiguous in global memory too.
      constexpr int KPC = 16 / (2 * T::ESZ);
      constexpr int CPR = TC_KP * T::ESZ / 16;      // 16-byte chunks per row
      constexpr int NCH = TC_M * CPR / TC_LOAD_THREADS;  // chunks per thread per stage
      const int lt = threadIdx.x - (TC_MMA_WARP + 1) * 32;
      const int tkv = 1 << g.tk;
      const bool kadj = g.nk > 0 && g.a_kpos[0] == 0;
      // lanes walk the k chunks of a row when A's lowest memory bit is a k bit,
      // else they walk rows; either way the swizzled stores are conflict-free
      const bool klanes = kadj;
      int64_t goff[NCH][KPC];   // offset of each complex of each chunk, -1 = padding
      int soff[NCH];
      bool cok[NCH];
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const int q = lt + j * TC_LOAD_THREADS;
        const int row = klanes ? q / CPR : q % TC_M;
        const int c = klanes ? q % CPR : q / TC_M;
        cok[j] = row < (1 << g.tm);
        soff[j] = tc_elem_off(row, c * KPC * 2, T::ESZ);
        const int64_t roff = deposit_hi((uint64_t)row, g.a_mpos, 0, g.tm);
#pragma unroll
        for (int i = 0; i < KPC; ++i) {
          const int k = c * KPC + i;
          goff[j][i] = (cok[j] && k < tkv) ? roff + deposit_hi((uint64_t)k, g.a_kpos, 0, g.tk) : -1;
        }
      }
      auto tile_base = [&](int64_t tile) -> const float2* {
        const TileIdx ti = tile_decode(tile, a);
        const int mt = own_mt(ti.mt), inst = ti.inst;
        return g.A + inst_offset(inst, g.a_istride, g.a_bpos, g.nb) + deposit_hi((uint64_t)mt, g.a_mpos, g.tm, g.nm);
      };
      int slot = 0;
      uint32_t ph = 0;
      if constexpr (MODE == TC_TF32) {
        bool ok = true;
        int64_t jt = 0;
        for (int64_t tile = seq_tile(0); tile >= 0 && ok; tile = seq_tile(++jt)) {
          const float2* At = tile_base(tile);
          const int kc0 = (int)(tile & (int64_t)(a.n_split - 1)) * kc_per;
          for (int kc = kc0; kc < kc0 + kc_per; ++kc) {
            const float2* Ak = At + deposit_hi((uint64_t)kc, g.a_kpos, g.tk, g.nk);
            uint8_t* sa = aring + slot * P::A_SLOT;
            if (!mbar_wait(smem_u32(&emptyA[slot]), ph ^ 1, abort_flag, a.err)) { ok = false; break; }
            {
              const bool v16 = kadj && ((reinterpret_cast<uintptr_t>(Ak) & 15) == 0);
#pragma unroll
              for (int j = 0; j < NCH; ++j) {
                if (!cok[j]) continue;
                if (v16 && goff[j][1] >= 0) {
                  cp_async16(smem_u32(sa + soff[j]), Ak + goff[j][0]);
                } else {
#pragma unroll
                  for (int i = 0; i < KPC; ++i)
                    if (goff[j][i] >= 0) cp_async8(smem_u32(sa + soff[j] + 8 * i), Ak + goff[j][i]);
                }
              }
            }
            cp_async_arrive_noinc(smem_u32(&fullA[slot]));
            if (++slot == na) {
              slot = 0;
              ph ^= 1;
            }
          }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
      } else {
        // BF16X3: the next slot's loads are in flight in registers while the
        // current one is split into hi/lo and stored
        float4 v0[NCH][KPC / 2], v1[NCH][KPC / 2];
        auto issue = [&](float4(&v)[NCH][KPC / 2], const float2* Ak) {
          const bool v16 = kadj && ((reinterpret_cast<uintptr_t>(Ak) & 15) == 0);
#pragma unroll
          for (int j = 0; j < NCH; ++j)
#pragma unroll
            for (int h = 0; h < KPC / 2; ++h) {
              const int64_t o0 = goff[j][2 * h], o1 = goff[j][2 * h + 1];
              if (v16 && o1 >= 0) {
                v[j][h] = __ldg(reinterpret_cast<const float4*>(Ak + o0));
              } else {
                const float2 x = o0 >= 0 ? __ldg(Ak + o0) : make_float2(0.f, 0.f);
                const float2 y = o1 >= 0 ? __ldg(Ak + o1) : make_float2(0.f, 0.f);
                v[j][h] = make_float4(x.x, x.y, y.x, y.y);
              }
            }
        };
        int64_t jt = 0;
        int64_t tile = seq_tile(0);
        int kc = tile >= 0 ? (int)(tile & (int64_t)(a.n_split - 1)) * kc_per : 0;
        const float2* At = tile >= 0 ? tile_base(tile) : g.A;
        const float2* An = At;     // base of the tile of the prefetched slot
        auto body = [&](float4(&vc)[NCH][KPC / 2], float4(&vn)[NCH][KPC / 2]) -> bool {
          int64_t ntile = tile, njt = jt;
          int nkc = kc + 1;
          if (nkc == (int)(tile & (int64_t)(a.n_split - 1)) * kc_per + kc_per) {
            ntile = seq_tile(++njt);
            nkc = ntile >= 0 ? (int)(ntile & (int64_t)(a.n_split - 1)) * kc_per : 0;
            if (ntile >= 0) An = tile_base(ntile);
          }
          if (ntile >= 0) issue(vn, An + deposit_hi((uint64_t)nkc, g.a_kpos, g.tk, g.nk));
          uint8_t* sa = aring + slot * P::A_SLOT;
          if (!mbar_wait(smem_u32(&emptyA[slot]), ph ^ 1, abort_flag, a.err)) return false;
          {
#pragma unroll
            for (int j = 0; j < NCH; ++j) {
              if (!cok[j]) continue;
              uint32_t hi[4], lo[4];
#pragma unroll
              for (int h = 0; h < KPC / 2; ++h) {
                const float4 x = vc[j][h];
                split_pair<MODE>(x.x * sc_a, x.y * sc_a, hi[2 * h], lo[2 * h]);
                split_pair<MODE>(x.z * sc_a, x.w * sc_a, hi[2 * h + 1], lo[2 * h + 1]);
              }
              *reinterpret_cast<uint4*>(sa + soff[j]) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
              *reinterpret_cast<uint4*>(sa + a_plane + soff[j]) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            }
          }
          fence_proxy_async();
          mbar_arrive(smem_u32(&fullA[slot]));
          if (++slot == na) {
            slot = 0;
            ph ^= 1;
          }
          if (ntile != tile) At = An;
          tile = ntile;
          jt = njt;
          kc = nkc;
          return true;
        };
        if (tile >= 0) issue(v0, At + deposit_hi((uint64_t)kc, g.a_kpos, g.tk, g.nk));
        while (tile >= 0) {
          if (!body(v0, v1) || tile < 0) break;
          if (!body(v1, v0)) break;
        }
      }
    }
  } else if (warp == TC_MMA_WARP) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0 && rank == 0) {
      // N of one MMA: all N' = 2 tn_c real columns (4M), or tn_c per product (3M);
      // M: 128 rows, or 256 for a pair (128 in each CTA)
      const int mma_n = CM == 4 ? ncp : a.tn_c;
      const uint32_t idesc = (1u << 4) | ((uint32_t)T::FMT << 7) | ((uint32_t)T::FMT << 10) |
                             ((uint32_t)(mma_n >> 3) << 17) | ((uint32_t)((PAIR ? 2 : 1) * TC_M >> 4) << 24);
      // operand descriptors of the ring bases: a slot, plane or K-step offset
      // is added to the 14-bit start-address field in 16-byte units (shared
      // addresses stay below 256 KB, so the field never carries)
      const uint32_t sbo = tc_sbo(T::ESZ);
      const uint32_t lay = T::ESZ == 4 ? 2u : 4u;
      const uint64_t dfa = smem_desc(smem_u32(aring), sbo, lay), dfb = smem_desc(smem_u32(bring), sbo, lay);
      const uint32_t da0 = (uint32_t)dfa, db0 = (uint32_t)dfb, dhi = (uint32_t)(dfa >> 32);
      const uint32_t a_step = (uint32_t)(P::A_SLOT >> 4), b_step = (uint32_t)(b_slot >> 4);
      const uint32_t ap = (uint32_t)(a_plane >> 4), bp = (uint32_t)(b_plane >> 4);
      // generic-proxy operand writes are ordered before the MMAs by their
      // writers, except the cp.async gathers of TF32 4M: fenced here
      const bool fence_a = MODE == TC_TF32 && CM == 4 && !a.a_tma;
      uint32_t da = da0, db = db0;
      int sa_i = 0, sb_i = 0, acc = 0;
      uint32_t pha = 0, aph = 0;
      bool ok = true;
      int64_t jt = 0;
      for (int64_t tile = seq_tile(0); tile >= 0 && ok; tile = seq_tile(++jt)) {
        // the accumulator set is drained (in both CTAs of a pair)
        if (!mbar_wait(smem_u32(&tempty[acc]), aph ^ 1, abort_flag, a.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * setw);
        for (int kc = 0; kc < kc_per; ++kc) {
          // the chunk's operands are in place (in both CTAs of a pair)
          if (!mbar_wait(smem_u32(&fullA[sa_i]), pha, abort_flag, a.err)) {
            ok = false;
            break;
          }
          if (fence_a) fence_proxy_async();
          tc_fence_after();
          auto mma = [&](uint32_t d, uint32_t adesc, uint32_t bdesc, uint32_t accumulate) {
            tc_mma<MODE, PAIR>(d, adesc, bdesc, dhi, idesc, accumulate);
          };
          // one MMA K step = 32 bytes of every plane row (2 descriptor units):
          // the step advances inside the swizzle atom
          if constexpr (CM == 4) {
#pragma unroll
            for (int j = 0; j < TC_KP * T::ESZ / 32; ++j) {
              const uint32_t ko = (uint32_t)(2 * j);
              const uint32_t first = (kc > 0 || j > 0) ? 1u : 0u;
              mma(d_tmem, da + ko, db + ko, first);
              if constexpr (MODE != TC_TF32) {   // hi*hi + hi*lo + lo*hi
                mma(d_tmem, da + ko, db + bp + ko, 1u);
                mma(d_tmem, da + ap + ko, db + ko, 1u);
              }
            }
          } else {
            // T1, T2, T3 in consecutive tn_c-column blocks of the accumulator set
            const uint32_t d1 = d_tmem, d2 = d_tmem + (uint32_t)a.tn_c, d3 = d_tmem + 2u * (uint32_t)a.tn_c;
            if constexpr (MODE == TC_TF32) {
              // planes [Ar | Ai], [As | -] against [Br | Bi], [Bs | 0]: two K steps of 8
#pragma unroll
              for (int j = 0; j < 2; ++j) {
                const uint32_t ko = (uint32_t)(2 * j);
                const uint32_t first = (kc > 0 || j > 0) ? 1u : 0u;
                mma(d1, da + ko, db + ko, first);
                mma(d2, da + 4u + ko, db + 4u + ko, first);
                mma(d3, da + ap + ko, db + bp + ko, first);
              }
            } else {
              // planes H = [Ar_hi | Ai_hi], L = [Ar_lo | Ai_lo], S = [As_hi | As_lo]
              const uint32_t first = kc > 0 ? 1u : 0u;
              const uint32_t H = da, L = da + ap, S = da + 2u * ap;
              const uint32_t BH = db, BL = db + bp, BS = db + 2u * bp;
              mma(d1, H, BH, first);
              mma(d1, H, BL, 1u);
              mma(d1, L, BH, 1u);
              mma(d2, H + 2u, BH + 2u, first);
              mma(d2, H + 2u, BL + 2u, 1u);
              mma(d2, L + 2u, BH + 2u, 1u);
              mma(d3, S, BS, first);
              mma(d3, S, BS + 2u, 1u);
              mma(d3, S + 2u, BS, 1u);
            }
          }
          tc_commit_g<PAIR>(smem_u32(&emptyA[sa_i]));
          da += a_step;
          if (++sa_i == na) {
            sa_i = 0;
            pha ^= 1;
            da = da0;
          }
          db += b_step;
          if (++sb_i == nbs) {
            sb_i = 0;
            db = db0;
          }
        }
        if (!ok) break;
        tc_commit_g<PAIR>(smem_u32(&tfull[acc]));
        if (++acc == a.n_acc) {
          acc = 0;
          aph ^= 1;
        }
      }
      // drain: every MMA issued so far completes before the CTA (or pair) frees
      // TMEM, also after an abort (within the limit)
      tc_commit_g<PAIR>(smem_u32(fin));
      mbar_wait<true>(smem_u32(fin), 0, abort_flag, a.err, 1000000000ull);
    } else if (PAIR && lane == 0) {
      // ---------------------------------------------------------------- pair relay (odd CTA)
      // Follows the MMA thread's order: per chunk, once this CTA's A and B'
      // slots are filled (its fullA), one arrival on the even CTA's fullA of
      // that slot; per tile after the first n_acc, once this CTA's epilogue has
      // drained the accumulator set, one arrival on the even CTA's tempty.  Each
      // arrival lands in the phase it completes: the even CTA's previous phase
      // of that barrier is over before this CTA's own one can complete (the
      // slot is refilled, the set drained, only after the even CTA's MMAs of
      // that previous phase).  The slots themselves are released by the MMAs'
      // commits, which reach both CTAs.
      const bool fence_a = MODE == TC_TF32 && CM == 4 && !a.a_tma;
      const uint32_t rA = mapa_cta(smem_u32(fullA), 0), rT = mapa_cta(smem_u32(tempty), 0);
      int sa_i = 0, acc = 0;
      uint32_t pha = 0, aph = 0;
      int64_t j = 0;
      bool ok = true;
      for (int64_t tile = seq_tile(0); tile >= 0 && ok; tile = seq_tile(++j)) {
        if (j >= a.n_acc) {
          if (!mbar_wait(smem_u32(&tempty[acc]), aph ^ 1, abort_flag, a.err)) break;
          mbar_arrive_remote(rT + 8u * (uint32_t)acc);
        }
        for (int kc = 0; kc < kc_per; ++kc) {
          if (!mbar_wait(smem_u32(&fullA[sa_i]), pha, abort_flag, a.err)) {
            ok = false;
            break;
          }
          if (fence_a) fence_proxy_async();
          mbar_arrive_remote(rA + 8u * (uint32_t)sa_i);
          if (++sa_i == na) {
            sa_i = 0;
            pha ^= 1;
          }
        }
        if (++acc == a.n_acc) {
          acc = 0;
          aph ^= 1;
        }
      }
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- epilogue
    const int row = warp * 32 + lane;
    // staged write-back: element e = lane + 32 i of the warp's 32 x 16 block;
    // e's bits (lane bits 0-4, i bits 5-8) sit at C positions epi_pos[] and at
    // staging-buffer strides w (row bit r: STRIDE 2^r, column bit c: 2^c), so
    // both addresses are sums of per-bit weights
    int sidx_l = 0;
    int64_t goff_l = 0;
    int ws[4] = {0, 0, 0, 0};
    int64_t wg[4] = {0, 0, 0, 0};
    if (a.epi_ok) {
      for (int t = 0; t < 9; ++t) {
        const int sl = a.epi_sel[t];
        const int w = (sl & 64) ? (1 << (sl & 63)) : (TC_EPI_STRIDE << (sl & 63));
        const int64_t o = (int64_t)1 << a.epi_pos[t];
        if (t < 5) {
          if ((lane >> t) & 1) {
            sidx_l += w;
            goff_l += o;
          }
        } else {
          ws[t - 5] = w;
          wg[t - 5] = o;
        }
      }
    }
    // the result's largest component, for its consumer's FP16 scaling (split-K
    // partials are not the result: the reduction records it)
    const bool track = g.amax_c != nullptr && a.n_split == 1;
    int acc = -1;
    uint32_t aph = 1;
    int64_t jt = 0;
    for (int64_t tile = seq_tile(0); tile >= 0; tile = seq_tile(++jt)) {
      if (++acc == a.n_acc) acc = 0;
      if (acc == 0) aph ^= 1;
      // warp-uniform decision: the TMEM loads and shuffles below need all 32 lanes
      if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&tfull[acc]), aph, abort_flag, a.err))) break;
      tc_fence_after();
      const TileIdx ti = tile_decode(tile, a);
      const int nt = ti.nt, mt = own_mt(ti.mt), inst = ti.inst;
      float2* Cb = a.n_split > 1 ? a.c_part + ti.s * a.c_part_stride : g.C;
      // the tile's base in C: its instance, m-tile and n-tile bits deposited at
      // their positions in C, one bit per lane, summed over the warp
      int64_t cb = (int64_t)inst * g.c_istride;
      {
        const int n_i = g.nb, n_m = g.nm - g.tm, n_all = g.nb + (g.nm - g.tm) + (g.nn - a.tnb);
        for (int b0 = 0; b0 < n_all; b0 += 32) {
          const int bi = b0 + lane;
          int64_t v = 0;
          if (bi < n_i) {
            if ((inst >> bi) & 1) v = (int64_t)1 << g.c_bpos[bi];
          } else if (bi < n_i + n_m) {
            if ((mt >> (bi - n_i)) & 1) v = (int64_t)1 << g.c_mpos[g.tm + bi - n_i];
          } else if (bi < n_all) {
            if ((nt >> (bi - n_i - n_m)) & 1) v = (int64_t)1 << g.c_npos[a.tnb + bi - n_i - n_m];
          }
#pragma unroll
          for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          cb += v;
        }
      }
      float2* C = Cb + cb;
      const bool row_ok = row < tmv;
      const int64_t crow = offCm[row];
      float am = 0.f;
      const uint32_t tl = tmem_base + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * setw);
      for (int c0 = 0; c0 < ncp; c0 += 32) {   // 16 complex columns per pass
        float v[32];
        if constexpr (CM == 4) {
          tmem_ld32(tl + (uint32_t)c0, v);
        } else {
          // Re = T1 - T2, Im = T3 - T1 - T2
          float t[48];
          const uint32_t cc = (uint32_t)(c0 / 2);
          tmem_ld16x3(tl + cc, tl + (uint32_t)a.tn_c + cc, tl + 2u * (uint32_t)a.tn_c + cc, t);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            v[2 * j] = t[j] - t[16 + j];
            v[2 * j + 1] = t[32 + j] - t[j] - t[16 + j];
          }
        }
        if constexpr (MODE == TC_FP16X3) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = v[j] * us_a * us_b;
        }
        if (track) {   // largest component of the valid columns of this row
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (row_ok && c0 / 2 + j < tnv) am = fmaxf(am, fmaxf(fabsf(v[2 * j]), fabsf(v[2 * j + 1])));
        }
        if (a.epi_ok) {
          // stage the warp's 32 x 16 block, then write it in C's memory order:
          // element e = lane + 32 i has its bits on C's lowest positions first
          float2* stg = epi_stage + warp * 32 * TC_EPI_STRIDE;
#pragma unroll
          for (int j = 0; j < 16; ++j) stg[lane * TC_EPI_STRIDE + j] = make_float2(v[2 * j], v[2 * j + 1]);
          __syncwarp();
          if (warp * 32 < tmv && c0 / 2 < tnv) {
            float2* base = C + offCm[warp * 32] + offCn[c0 / 2] + goff_l;
            const float2* sbase = stg + sidx_l;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              int si = 0;
              int64_t gi = 0;
#pragma unroll
              for (int j = 0; j < 4; ++j)
                if ((i >> j) & 1) {
                  si += ws[j];
                  gi += wg[j];
                }
              base[gi] = sbase[si];
            }
          }
          __syncwarp();
        } else if (row_ok) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = c0 / 2 + j;
            if (n < tnv) C[crow + offCn[n]] = make_float2(v[2 * j], v[2 * j + 1]);
          }
        }
      }
      if (track) amax_update(g.amax_c, am);   // all 32 lanes of the warp
      tc_fence_before();
      mbar_arrive(smem_u32(&tempty[acc]));
    }
  }
  tc_fence_before();
  __syncthreads();
  // neither CTA of a pair leaves (or frees TMEM) while the other may still
  // reach its shared memory: the even CTA arrives here after its MMAs drained
  if constexpr (PAIR) cluster_sync_all();
  if (warp == TC_MMA_WARP) {
    tc_fence_after();
    if constexpr (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TC_TMEM_COLS)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TC_TMEM_COLS)
                   : "memory");
  }
}

}  // namespace tnx
