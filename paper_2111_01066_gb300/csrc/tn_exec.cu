// Device executor: the slice loop of a plan on one GPU, the XEB reduction, and
// the standalone kernel entry points of the C ABI.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <array>
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "k_misc.cuh"
#include "k_simt.cuh"
#include "k_tc.cuh"
#include "kernels_common.cuh"
#include "tn_internal.h"

namespace tnx {

#define CK(x)                                                                          \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess) fail(TN_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ------------------------------------------------------------------ kernel table
enum KernelId {
  K_SIMT_64x64 = 0,   // TM 64, TN 64, TK 8
  K_SIMT_128x16 = 1,  // TM 128, TN 16, TK 16
  K_SIMT_256x4 = 2,   // TM 256, TN 4, TK 16
  K_TC_TF32 = 3,      // tcgen05 kind::tf32, tile 128 x (<=128 complex), k chunk 16
  K_TC_BF16X3 = 4,    // tcgen05 kind::f16 bf16 hi/lo split
  K_TC_TF32_3M = 5,   // the same with 3M products (three accumulators per tile)
  K_TC_BF16X3_3M = 6,
  K_TC_FP16X3 = 7,    // tcgen05 kind::f16 fp16 hi/lo split, operands scaled by powers of two
  K_TC_FP16X3_3M = 8,
  K_COUNT
};
struct KernelCfg {
  int tm, tn, tk;  // log2 tile extents
};
static const KernelCfg kCfg[K_COUNT] = {{6, 6, 3}, {7, 4, 4}, {8, 2, 4}, {7, 7, 4}, {7, 7, 4}, {7, 7, 4}, {7, 7, 4}, {7, 7, 4}, {7, 7, 4}};

static int pick_simt(const StepDesc& d) {
  if (d.nn >= 5 && d.nm >= 5) return K_SIMT_64x64;
  if (d.nn >= 3) return K_SIMT_128x16;
  return K_SIMT_256x4;
}

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  }
  return n;
}

// Tile decode tables: the tile's bits in ascending memory position.
static GemmArgs make_args(const StepDesc& d, int kid, const float2* A, const float2* B, float2* C,
                          int32_t n_inst, int64_t a_istride = 0, int64_t b_istride = 0,
                          int64_t c_istride = 0, int tn_log = -1) {
  GemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.A = A;
  g.B = B;
  g.C = C;
  g.a_istride = a_istride;
  g.b_istride = b_istride;
  g.c_istride = c_istride;
  g.n_inst = n_inst;
  g.nb = d.nb;
  g.nm = d.nm;
  g.nk = d.nk;
  g.nn = d.nn;
  std::memcpy(g.a_bpos, d.a_bpos, KMAXB);
  std::memcpy(g.b_bpos, d.b_bpos, KMAXB);
  std::memcpy(g.c_bpos, d.c_bpos, KMAXB);
  const KernelCfg& k = kCfg[kid];
  g.tm = std::min(k.tm, d.nm);
  g.tk = std::min(k.tk, d.nk);
  g.tn = std::min(tn_log >= 0 ? tn_log : k.tn, d.nn);
  std::memcpy(g.a_mpos, d.a_mpos, KMAXR);
  std::memcpy(g.a_kpos, d.a_kpos, KMAXR);
  std::memcpy(g.b_kpos, d.b_kpos, KMAXR);
  std::memcpy(g.b_npos, d.b_npos, KMAXR);
  std::memcpy(g.c_mpos, d.c_mpos, KMAXR);
  std::memcpy(g.c_npos, d.c_npos, KMAXR);
  std::vector<std::pair<int, int>> ta, tb;  // (position, sel)
  for (int i = 0; i < g.tm; ++i) ta.push_back({d.a_mpos[i], i});
  for (int j = 0; j < g.tk; ++j) ta.push_back({d.a_kpos[j], j | 64});
  for (int j = 0; j < g.tk; ++j) tb.push_back({d.b_kpos[j], j | 64});
  for (int i = 0; i < g.tn; ++i) tb.push_back({d.b_npos[i], i});
  std::sort(ta.begin(), ta.end());
  std::sort(tb.begin(), tb.end());
  if ((int)ta.size() > KTB || (int)tb.size() > KTB) fail(TN_ERR_UNSUPPORTED, "tile too large");
  g.a_tbits = (int)ta.size();
  g.b_tbits = (int)tb.size();
  for (size_t t = 0; t < ta.size(); ++t) {
    g.a_tpos[t] = (int8_t)ta[t].first;
    g.a_tsel[t] = (int8_t)ta[t].second;
  }
  for (size_t t = 0; t < tb.size(); ++t) {
    g.b_tpos[t] = (int8_t)tb[t].first;
    g.b_tsel[t] = (int8_t)tb[t].second;
  }
  return g;
}

static void launch_simt(const GemmArgs& g, int kid, cudaStream_t s) {
  if (g.n_inst <= 0) return;
  const int64_t gx = (int64_t)1 << (g.nm - g.tm);
  const int64_t gy = (int64_t)1 << (g.nn - g.tn);
  if (gx > 0x7fffffff || gy > 65535) fail(TN_ERR_UNSUPPORTED, "GEMM grid too large");
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)std::min<int32_t>(g.n_inst, 65535));
  switch (kid) {
    case K_SIMT_64x64:
      k_cgemm_simt<64, 64, 8, 4, 4><<<grid, 256, 0, s>>>(g);
      break;
    case K_SIMT_128x16:
      k_cgemm_simt<128, 16, 16, 4, 2><<<grid, 256, 0, s>>>(g);
      break;
    case K_SIMT_256x4:
      k_cgemm_simt<256, 4, 16, 4, 1><<<grid, 256, 0, s>>>(g);
      break;
    default:
      fail(TN_ERR_UNSUPPORTED, "kernel variant not built");
  }
}

// One step ready to launch: GEMM arguments, tensor-core tiling, B' workspace
// size, and the tensor map of A when its tiles are fetched by TMA.
struct StepLaunch {
  int kid = 0;
  GemmArgs g;
  TcArgs tc;
  CUtensorMap tma;   // 64-byte aligned by its own declaration
  int64_t ws_bytes = 0;
  int64_t split_off = 0;   // split-K partials inside the workspace
  int64_t c_total = 0;     // elements of C (all instances)
  int smem = 0;
  // B' images built ahead of the chunks (the step's B depends on no slice):
  // built by the prologue of class bimg_cls (0 once per plan, 2 once per
  // batch) into bimg_own; null: built with every launch in the workspace
  uint8_t* bimg_own = nullptr;
  int bimg_cls = -1;
};

static bool is_tc(int kid) { return kid >= K_TC_TF32 && kid <= K_TC_FP16X3_3M; }
static bool tc_is_3m(int kid) { return kid == K_TC_TF32_3M || kid == K_TC_BF16X3_3M || kid == K_TC_FP16X3_3M; }
struct TcGeom {   // the plane geometry of TcPl<MODE, CM> for a kernel id
  int planes, rows_per_col, a_slot, min_tn_c, esz;
};
static TcGeom tc_geom(int kid) {
  switch (kid) {
    case K_TC_TF32:
      return {TcPl<TC_TF32, 4>::PLANES, TcPl<TC_TF32, 4>::ROWS_PER_COL, TcPl<TC_TF32, 4>::A_SLOT,
              TcPl<TC_TF32, 4>::MIN_TN_C, 4};
    case K_TC_BF16X3:
      return {TcPl<TC_BF16X3, 4>::PLANES, TcPl<TC_BF16X3, 4>::ROWS_PER_COL, TcPl<TC_BF16X3, 4>::A_SLOT,
              TcPl<TC_BF16X3, 4>::MIN_TN_C, 2};
    case K_TC_TF32_3M:
      return {TcPl<TC_TF32, 3>::PLANES, TcPl<TC_TF32, 3>::ROWS_PER_COL, TcPl<TC_TF32, 3>::A_SLOT,
              TcPl<TC_TF32, 3>::MIN_TN_C, 4};
    case K_TC_BF16X3_3M:
      return {TcPl<TC_BF16X3, 3>::PLANES, TcPl<TC_BF16X3, 3>::ROWS_PER_COL, TcPl<TC_BF16X3, 3>::A_SLOT,
              TcPl<TC_BF16X3, 3>::MIN_TN_C, 2};
    case K_TC_FP16X3:
      return {TcPl<TC_FP16X3, 4>::PLANES, TcPl<TC_FP16X3, 4>::ROWS_PER_COL, TcPl<TC_FP16X3, 4>::A_SLOT,
              TcPl<TC_FP16X3, 4>::MIN_TN_C, 2};
    default:
      return {TcPl<TC_FP16X3, 3>::PLANES, TcPl<TC_FP16X3, 3>::ROWS_PER_COL, TcPl<TC_FP16X3, 3>::A_SLOT,
              TcPl<TC_FP16X3, 3>::MIN_TN_C, 2};
  }
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// A can be fetched by TMA when it is stored as [its k bits in order, then at
// least 128 rows of m bits in order]: a row-major matrix per dimension-2 index.
// a_bits = log2 of A's elements over one linear instance; n_lin = linear instances.
static void setup_tma(StepLaunch& L, int a_bits, int64_t n_lin) {
  const GemmArgs& g = L.g;
  TcArgs& t = L.tc;
  t.a_tma = 0;
  // tiles of 2^tm rows (tm <= 7; a 128-row MMA tile whose rows past 2^tm the epilogue drops)
  if (g.nk < 4 || g.tm < 3 || g.tm > 7 || (reinterpret_cast<uintptr_t>(g.A) & 15)) return;
  for (int j = 0; j < g.nk; ++j)
    if (g.a_kpos[j] != j) return;
  int nmw = 0;
  while (nmw < g.nm && g.a_mpos[nmw] == g.nk + nmw) ++nmw;
  if (nmw < g.tm) return;
  const int hi_shift = g.nk + nmw;
  if (a_bits < hi_shift) return;
  const uint64_t dim2 = ((uint64_t)1 << (a_bits - hi_shift)) * (uint64_t)n_lin;
  if (dim2 > ((uint64_t)1 << 31)) return;
  auto enc = tensor_map_encoder();
  if (!enc) return;
  cuuint64_t dims[3] = {(cuuint64_t)2 << g.nk, (cuuint64_t)1 << nmw, (cuuint64_t)dim2};
  cuuint64_t strides[2] = {((cuuint64_t)1 << g.nk) * 8, ((cuuint64_t)1 << hi_shift) * 8};
  cuuint32_t box[3] = {(cuuint32_t)TC_KP, (cuuint32_t)1u << g.tm, 1};
  cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(&L.tma, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(g.A), dims, strides, box,
                         es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return;
  t.a_tma = 1;
  t.a_box_bytes = (TC_KP * 4) << g.tm;
  t.nmw = nmw;
  t.hi_shift = hi_shift;
  t.c2_inst_mul = n_lin > 1 ? ((int64_t)1 << (a_bits - hi_shift)) : 0;
}

// epi_mode: -1 chooses the write-back by the coalesced run lengths, 0 forces
// direct per-column stores, 1 the staged order (where the tile allows it)
// b_slots: B' ring slots (<= 0: 4 for slots up to 16 KB, else 3; at most
// TC_MAX_B; the rest of the shared-memory budget goes to A slots)
// pair_mode: SM pairs (cta_group::2, two m tiles per work unit, half of B' per
// CTA) where the step allows them -- 4M products and at least two full 128-row
// m tiles: -1 or 1 uses them there, 0 never
static bool pair_ok(const GemmArgs& g, int kid) { return !tc_is_3m(kid) && g.tm == 7 && g.nm - g.tm >= 1; }
static StepLaunch make_launch(const GemmArgs& g, int kid, int a_bits, int64_t n_lin, int64_t c_total = 0,
                              bool allow_split = false, int epi_mode = -1,
                              int64_t split_cap_bytes = (int64_t)256 << 20, int b_slots = 0, int pair_mode = -1) {
  StepLaunch L;
  L.kid = kid;
  L.g = g;
  std::memset(&L.tc, 0, sizeof(L.tc));
  std::memset(&L.tma, 0, sizeof(L.tma));
  if (!is_tc(kid)) return L;
  TcArgs& t = L.tc;
  t.g = g;
  t.tnb = g.tn;
  const TcGeom geo = tc_geom(kid);
  t.tn_c = std::max(geo.min_tn_c, 1 << g.tn);
  t.pair = (pair_mode != 0 && pair_ok(g, kid)) ? 1 : 0;
  t.n_mt = 1 << (g.nm - g.tm - t.pair);
  t.n_nt = 1 << (g.nn - g.tn);
  t.n_kc = 1 << (g.nk - g.tk);
  t.n_tiles = (int64_t)g.n_inst * t.n_mt * t.n_nt;
  const int b_plane = tc_plane_bytes(geo.rows_per_col * t.tn_c, geo.esz);
  const int npl = geo.planes;
  L.ws_bytes = (int64_t)g.n_inst * t.n_nt * t.n_kc * npl * b_plane;
  // split-K when the output tiles cannot fill the SMs and the k loop is long
  // (a pair's work unit occupies two SMs)
  const int64_t unit_sms = 1 + t.pair;
  t.n_split = 1;
  if (allow_split && c_total > 0 && t.n_tiles * unit_sms < sm_count() && t.n_kc >= 8) {
    int sp = 1;
    // enough tiles for several waves (tail below ~15%), each split >= 4 k chunks
    while (sp < 32 && t.n_tiles * unit_sms * sp * 2 <= 8 * (int64_t)sm_count() && t.n_kc / (sp * 2) >= 4) sp *= 2;
    if (sp > 1 && (int64_t)sp * c_total * 8 <= split_cap_bytes) {
      t.n_split = sp;
      t.c_part_stride = c_total;
      L.split_off = (L.ws_bytes + 255) / 256 * 256;
      L.ws_bytes = L.split_off + (int64_t)sp * c_total * 8;
      L.c_total = c_total;
    }
  }
  t.n_tiles *= t.n_split;
  t.ls_split = __builtin_ctz((unsigned)t.n_split);
  t.ls_nt = g.nn - g.tn;
  t.ls_mt = g.nm - g.tm - t.pair;
  // the n tiles of one A block back to back on the same SM (pair), so that the
  // block's later reads hit L2: when the A blocks in flight on all SMs fit half
  // of L2 (else they evict each other between reads, while in index order the
  // n tiles of a block run at the same time on neighbouring SMs) and there are
  // at least 8 blocks per SM (pair), so that the coarser units leave no long tail
  const int64_t units = t.pair ? sm_count() / 2 : sm_count();
  const double a_block_bytes = 8.0 * TC_M * (1 + t.pair) * std::ldexp(1.0, g.nk);
  t.nt_inner = (t.n_nt > 1 && (t.n_tiles >> t.ls_nt) >= 8 * units &&
                units * a_block_bytes <= 64.0 * (1 << 20))
                   ? 1
                   : 0;
  t.ls_kc = g.nk - g.tk;
  setup_tma(L, a_bits, n_lin);
  // epilogue write order: a warp's rows are m bits 0-4, a chunk's 16 columns n bits 0-3
  t.epi_ok = 0;
  if (g.tm >= 5 && g.tn >= 4) {
    std::vector<std::pair<int, int>> bits;
    for (int i = 0; i < 5; ++i) bits.push_back({g.c_mpos[i], i});
    for (int j = 0; j < 4; ++j) bits.push_back({g.c_npos[j], j | 64});
    std::sort(bits.begin(), bits.end());
    for (int t2 = 0; t2 < 9; ++t2) {
      t.epi_pos[t2] = (int8_t)bits[t2].first;
      t.epi_sel[t2] = (int8_t)bits[t2].second;
    }
    // direct per-column stores write runs of 2^run_d elements (C's lowest
    // positions hold row bits 0, 1, ... in order); the staged order writes runs
    // of 2^run_s (C's lowest positions among the block's 9 bits).  Runs of 4+
    // elements fill whole 32-byte sectors, so stage only below that
    int run_d = 0, run_s = 0;
    while (run_d < 5 && g.c_mpos[run_d] == run_d) ++run_d;
    while (run_s < 5 && bits[run_s].first == run_s) ++run_s;
    t.epi_ok = epi_mode >= 0 ? epi_mode : (run_s > run_d && run_d < 2 ? 1 : 0);
  }
  // rings: B' slots first (3, or 4 when small), the rest of the shared memory
  // to A slots: up to the 227 KB opt-in, less the barriers, the alignment slack
  // and the write-back staging (only when the staged order is used); a pair's
  // CTA holds half of every B' plane
  const int b_slot = npl * (t.pair ? b_plane / 2 : b_plane);
  const int epi_bytes = t.epi_ok ? TC_EPI_BYTES : 0;
  const int budget = TC_MAX_SMEM - 4096 - 1024 - epi_bytes;
  t.nbs = b_slots > 0 ? std::min(b_slots, TC_MAX_B) : (b_slot <= 16384 ? 4 : 3);
  t.na = std::min(TC_MAX_A, (budget - t.nbs * b_slot) / geo.a_slot);
  // A by tensor-map loads converted in place: the two converter groups take
  // alternate k chunks, and chunk q sits in A slot q % na.  An even na keeps
  // every slot with one group, which then waits for the slot's phases strictly
  // in order; with an odd na a group could wait for phase u of a slot before the
  // other group's phase u - 1 had landed, and a parity wait cannot tell the two
  // apart (it would pass on the stale phase and convert the wrong data).
  const bool converters = t.a_tma && (tc_is_3m(kid) || kid != K_TC_TF32);
  if (converters) t.na &= ~1;
  if (t.na < 2) fail(TN_ERR_UNSUPPORTED, "tensor-core rings do not fit shared memory");
  t.nbs = std::min(t.nbs, t.na);   // B' slots are released through the A slots' barriers
  // arrivals on an A slot: the TMA itself (TF32 4M), one converter group (TMA otherwise), all loaders
  t.fa_count = (t.a_tma && kid == K_TC_TF32) ? 1 : (t.a_tma ? TC_LOAD_THREADS / 2 : TC_LOAD_THREADS);
  // as many accumulator sets as fit the 512 TMEM columns (at most 8): narrow
  // tiles let the MMAs run several tiles ahead of the epilogue
  t.n_acc = std::max(1, std::min(TC_MAX_ACC, TC_TMEM_COLS / ((tc_is_3m(kid) ? 3 : 2) * t.tn_c)));
  L.smem = std::max(t.na * geo.a_slot + t.nbs * b_slot + 4096 + epi_bytes + 1024, TC_MIN_SMEM);
  return L;
}

// SM pairs of a tensor-core kernel that can be resident at once (one pair per
// two SMs when the device fits them all), queried once per kernel and device
template <int MODE, bool PAIR>
static int pair_clusters() {
  static std::atomic<int> cached[64];
  int dev = 0;
  CK(cudaGetDevice(&dev));
  const int slot = dev < 64 ? dev : 63;
  int n = cached[slot].load(std::memory_order_acquire);
  if (n > 0) return n;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * (sm_count() / 2));
  cfg.blockDim = dim3(TC_THREADS);
  cfg.dynamicSmemBytes = TC_MAX_SMEM;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int q = 0;
  if (cudaOccupancyMaxActiveClusters(&q, k_cgemm_tc<MODE, 4, PAIR>, &cfg) != cudaSuccess || q <= 0) {
    cudaGetLastError();
    q = sm_count() / 2;
  }
  n = std::min(q, sm_count() / 2);
  cached[slot].store(n, std::memory_order_release);
  return n;
}

// The B' images of a tensor-core step into t.bimg: one CTA per image block at a time.
template <int MODE, int CM>
static void launch_prep(const TcArgs& t, cudaStream_t s) {
  const int64_t n_blocks = (int64_t)t.g.n_inst * t.n_nt * t.n_kc;
  const int pgrid = (int)std::max<int64_t>(1, std::min<int64_t>(n_blocks, (int64_t)sm_count() * 16));
  if constexpr (CM == 4)
    k_tc_prep_b<MODE><<<pgrid, 256, 0, s>>>(t);
  else
    k_tc_prep_b3<MODE><<<pgrid, 256, 0, s>>>(t);
}
static void launch_prep_kid(const TcArgs& t, int kid, cudaStream_t s) {
  switch (kid) {
    case K_TC_TF32:
      launch_prep<TC_TF32, 4>(t, s);
      break;
    case K_TC_BF16X3:
      launch_prep<TC_BF16X3, 4>(t, s);
      break;
    case K_TC_TF32_3M:
      launch_prep<TC_TF32, 3>(t, s);
      break;
    case K_TC_BF16X3_3M:
      launch_prep<TC_BF16X3, 3>(t, s);
      break;
    case K_TC_FP16X3:
      launch_prep<TC_FP16X3, 4>(t, s);
      break;
    default:
      launch_prep<TC_FP16X3, 3>(t, s);
      break;
  }
}

template <int MODE, int CM, bool PAIR>
static void launch_tc(const TcArgs& t, const StepLaunch& L, int grid, cudaStream_t s) {
  if (!L.bimg_own) launch_prep<MODE, CM>(t, s);   // else built ahead by a prologue
  // the shared-memory opt-in is a per-device function attribute: one bit per
  // device (ids < 64) records that it was set there; two threads racing on the
  // same bit both set the same value, which is harmless
  static std::atomic<uint64_t> attr_set{0};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  const uint64_t bit = dev < 64 ? (1ULL << dev) : 0;
  if (!bit || !(attr_set.load(std::memory_order_acquire) & bit)) {
    CK(cudaFuncSetAttribute(k_cgemm_tc<MODE, CM, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_MAX_SMEM));
    attr_set.fetch_or(bit, std::memory_order_acq_rel);
  }
  if constexpr (PAIR) {
    // clusters of two CTAs, each pair persistent over the work units
    const int clusters = (int)std::min<int64_t>(t.n_tiles, pair_clusters<MODE, PAIR>());
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * clusters);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = L.smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, k_cgemm_tc<MODE, CM, PAIR>, t, L.tma));
  } else {
    k_cgemm_tc<MODE, CM, PAIR><<<grid, TC_THREADS, L.smem, s>>>(t, L.tma);
  }
}

static void launch_step(StepLaunch& L, uint8_t* ws, int32_t* err, cudaStream_t s) {
  if (L.g.amax_c) CK(cudaMemsetAsync(L.g.amax_c, 0, sizeof(float), s));   // the result's maximum, recorded anew
  if (!is_tc(L.kid)) {
    launch_simt(L.g, L.kid, s);
    return;
  }
  TcArgs t = L.tc;
  t.bimg = L.bimg_own ? L.bimg_own : ws;
  t.err = err;
  if (t.n_split > 1) t.c_part = reinterpret_cast<float2*>(ws + L.split_off);
  if (t.n_tiles <= 0) return;
  const int grid = (int)std::min<int64_t>(t.n_tiles, sm_count());
  switch (L.kid) {
    case K_TC_TF32:
      if (t.pair)
        launch_tc<TC_TF32, 4, true>(t, L, grid, s);
      else
        launch_tc<TC_TF32, 4, false>(t, L, grid, s);
      break;
    case K_TC_BF16X3:
      if (t.pair)
        launch_tc<TC_BF16X3, 4, true>(t, L, grid, s);
      else
        launch_tc<TC_BF16X3, 4, false>(t, L, grid, s);
      break;
    case K_TC_TF32_3M:
      launch_tc<TC_TF32, 3, false>(t, L, grid, s);
      break;
    case K_TC_BF16X3_3M:
      launch_tc<TC_BF16X3, 3, false>(t, L, grid, s);
      break;
    case K_TC_FP16X3:
      if (t.pair)
        launch_tc<TC_FP16X3, 4, true>(t, L, grid, s);
      else
        launch_tc<TC_FP16X3, 4, false>(t, L, grid, s);
      break;
    default:
      launch_tc<TC_FP16X3, 3, false>(t, L, grid, s);
      break;
  }
  if (t.n_split > 1) {
    const int rb = (int)std::min<int64_t>((L.c_total + 255) / 256, (int64_t)sm_count() * 8);
    k_split_reduce<<<rb, 256, 0, s>>>(t.c_part, t.n_split, t.c_part_stride, t.g.C, L.c_total, t.g.amax_c);
  }
}

// ------------------------------------------------------------------ plan device state
struct DeviceState {
  int device = -1;
  float2* arena = nullptr;
  float2* leaf_data = nullptr;
  LeafDesc* leaf_desc = nullptr;
  ChunkParam* params = nullptr;
  size_t params_cap = 0;
  unsigned* counter = nullptr;
  int32_t* err = nullptr;
  uint8_t* ws = nullptr;
  int64_t ws_bytes = 0;           // capacity of ws
  double2* root_part = nullptr;   // [groups][2^k] partial slice sums
  float* amax = nullptr;          // FP16X3: largest component of every node (leaves, then steps)
  int root_groups = 1;
  std::vector<StepLaunch> launches;
  // groups of small independent steps (StepDesc::group): per group, the steps
  // [first, end) and the launches that run them -- one multi-step launch for
  // all its CUDA-core steps (each block with its step's tiling), single
  // launches for its tensor-core steps; rebuilt whenever the kernels are
  // chosen again
  struct GroupRun {
    int first = 0, end = 0;
    std::vector<int> singles;                  // steps launched alone
    struct Multi {
      int blocks = 0, n = 0;
      GemmArgs* args = nullptr;                // device: n GemmArgs
      int32_t* start = nullptr;                // device: n + 1 block offsets
      int8_t* tiling = nullptr;                // device: n CUDA-core tilings (kernel ids 0-2)
      std::vector<float*> amax;                // FP16X3: result maxima to clear first
    };
    std::vector<Multi> multi;
  };
  std::vector<GroupRun> groups;
  std::vector<int> group_at;                   // per step: its group run's index, or -1
  uint8_t* group_buf = nullptr;                // device memory of every Multi's arrays
  std::vector<uint8_t*> own_imgs;              // B' images built ahead of the chunks (StepLaunch::bimg_own)
  cudaEvent_t done = nullptr;
  bool have_done = false;
  // the chunk's launch sequence as one CUDA graph, captured after the first
  // eager chunk; every kernel reads its chunk parameters from device memory
  cudaGraphExec_t graph = nullptr;
  bool graph_failed = false;
  bool eager_done = false;
  // prologues: steps whose result depends on no slice run once per plan
  // (dependence flags 0) or once per batch bitstring (flags 2); their results
  // that later steps read sit in the arena's persistent pool
  bool pro0_done = false;
  bool pro2_valid = false;
  uint64_t pro2_bits = 0;
};

static int tc_kernel(int precision, int cmult) {
  if (precision == TN_PREC_TF32) return cmult == 3 ? K_TC_TF32_3M : K_TC_TF32;
  if (precision == TN_PREC_FP16X3) return cmult == 3 ? K_TC_FP16X3_3M : K_TC_FP16X3;
  return cmult == 3 ? K_TC_BF16X3_3M : K_TC_BF16X3;
}
// Tensor-core kernels (4M or 3M products) for every step with enough work in
// the TF32 / BF16X3 / FP16X3 modes; tiny steps (and the FP32 mode) on the CUDA
// cores, which always form 4M products in FP32.
static int pick_kernel(int precision, int cmult, const StepDesc& d) {
  if (precision == TN_PREC_FP32) return pick_simt(d);
  const int work = d.nm + d.nk + d.nn + d.nb;
  if (work < 20 || d.nm < 4) return pick_simt(d);
  return tc_kernel(precision, cmult);
}

// Launch arguments of plan step d for kernel kid; FP16X3 plans also get the
// maxima of the step's operands (to scale them) and of its result (to record).
static GemmArgs step_args(const DeviceState& ds, const StepDesc& d, int kid, int tn_log = -1) {
  GemmArgs g = make_args(d, kid, ds.arena + d.a_off, ds.arena + d.b_off, ds.arena + d.c_off, 1 << d.nb, 0, 0, 0,
                         tn_log);
  if (ds.amax) {
    g.amax_a = ds.amax + d.a_node;
    g.amax_b = ds.amax + d.b_node;
    g.amax_c = ds.amax + d.c_node;
  }
  return g;
}

static void launch_simt_multi(const DeviceState::GroupRun::Multi& m, cudaStream_t s) {
  for (float* am : m.amax) CK(cudaMemsetAsync(am, 0, sizeof(float), s));
  k_cgemm_simt_multi<<<m.blocks, 256, 0, s>>>(m.args, m.start, m.tiling, m.n);
}

// Dependence flags of a node (bit 0: on the slice id, bit 1: on the closed
// output bits): a step's own flags; a leaf's from the wires its select fixes
// and the slice bits it carries as batch bits.
static int node_flags(const Plan& p, int node) {
  const int nl = (int)p.leaves.size();
  if (node >= nl) return p.steps[node - nl].dep_flags;
  const LeafDesc& lf = p.leaves[node];
  int f = lf.bmask ? 1 : 0;
  for (int t = 0; t < lf.nfixed; ++t) f |= lf.fixed_kind[t] == 0 ? 1 : 2;
  return f;
}

// B' images of per-chunk tensor-core steps whose B depends on no slice: one
// buffer each, built by the prologue of B's class (once per plan, or once per
// batch bitstring) instead of with every chunk.  Where a buffer cannot be had
// the step keeps building its images per launch.
static void setup_hoisted(Plan& p, DeviceState& ds) {
  for (uint8_t* b : ds.own_imgs) cudaFree(b);
  ds.own_imgs.clear();
  for (size_t i = 0; i < p.steps.size(); ++i) {
    StepLaunch& L = ds.launches[i];
    L.bimg_own = nullptr;
    L.bimg_cls = -1;
    const StepDesc& d = p.steps[i];
    if (!is_tc(L.kid) || !(d.dep_flags & 1)) continue;
    const int bf = node_flags(p, d.b_node);
    if (bf & 1) continue;
    const int64_t img = L.tc.n_split > 1 ? L.split_off : L.ws_bytes;
    uint8_t* buf = nullptr;
    if (img <= 0 || cudaMalloc(&buf, (size_t)img) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    ds.own_imgs.push_back(buf);
    L.bimg_own = buf;
    L.bimg_cls = bf;
  }
}

// Group runs from the plan's step groups and the kernels chosen so far.
static void build_groups(Plan& p, DeviceState& ds) {
  if (ds.group_buf) {
    CK(cudaFree(ds.group_buf));
    ds.group_buf = nullptr;
  }
  ds.groups.clear();
  ds.group_at.assign(p.steps.size(), -1);
  std::vector<std::pair<size_t, std::vector<int>>> pending;   // (group run, steps) of each Multi
  for (size_t i = 0; i < p.steps.size();) {
    const int gid = p.steps[i].group;
    size_t j = i + 1;
    if (gid >= 0)
      while (j < p.steps.size() && p.steps[j].group == gid) ++j;
    if (gid < 0 || j - i < 2) {
      i = j;
      continue;
    }
    DeviceState::GroupRun gr;
    gr.first = (int)i;
    gr.end = (int)j;
    std::vector<int> simt;
    for (size_t t = i; t < j; ++t) {
      if (is_tc(ds.launches[t].kid)) gr.singles.push_back((int)t);
      else simt.push_back((int)t);
    }
    if (simt.size() == 1) gr.singles.push_back(simt[0]);
    if (simt.size() >= 2) {
      DeviceState::GroupRun::Multi m;
      m.n = (int)simt.size();
      gr.multi.push_back(m);
      pending.push_back({ds.groups.size(), simt});
    }
    for (size_t t = i; t < j; ++t) ds.group_at[t] = (int)ds.groups.size();
    ds.groups.push_back(gr);
    i = j;
  }
  if (pending.empty()) return;
  // one device buffer: every Multi's GemmArgs, then its block offsets
  size_t bytes = 0;
  for (auto& pm : pending) {
    bytes = (bytes + 255) / 256 * 256 + sizeof(GemmArgs) * pm.second.size();
    bytes = (bytes + 15) / 16 * 16 + sizeof(int32_t) * (pm.second.size() + 1);
    bytes += pm.second.size();   // tilings
  }
  std::vector<uint8_t> host(bytes, 0);
  CK(cudaMalloc(&ds.group_buf, bytes));
  size_t off = 0;
  std::vector<size_t> next_multi(ds.groups.size(), 0);
  for (auto& pm : pending) {
    auto& m = ds.groups[pm.first].multi[next_multi[pm.first]++];
    off = (off + 255) / 256 * 256;
    const size_t args_off = off;
    off += sizeof(GemmArgs) * pm.second.size();
    off = (off + 15) / 16 * 16;
    const size_t start_off = off;
    off += sizeof(int32_t) * (pm.second.size() + 1);
    const size_t tiling_off = off;
    off += pm.second.size();
    int32_t blocks = 0;
    for (size_t q = 0; q < pm.second.size(); ++q) {
      const GemmArgs& g = ds.launches[pm.second[q]].g;
      std::memcpy(host.data() + args_off + q * sizeof(GemmArgs), &g, sizeof(GemmArgs));
      host[tiling_off + q] = (uint8_t)ds.launches[pm.second[q]].kid;   // K_SIMT_* are 0..2
      const int64_t nb = ((int64_t)1 << (g.nm - g.tm)) * ((int64_t)1 << (g.nn - g.tn)) *
                         std::min<int64_t>(g.n_inst, 65535);
      if (blocks + nb > 0x7fffffff) fail(TN_ERR_UNSUPPORTED, "step group grid too large");
      std::memcpy(host.data() + start_off + q * sizeof(int32_t), &blocks, sizeof(int32_t));
      blocks += (int32_t)nb;
      if (g.amax_c) m.amax.push_back(g.amax_c);
    }
    std::memcpy(host.data() + start_off + pm.second.size() * sizeof(int32_t), &blocks, sizeof(int32_t));
    m.blocks = blocks;
    m.args = reinterpret_cast<GemmArgs*>(ds.group_buf + args_off);
    m.start = reinterpret_cast<int32_t*>(ds.group_buf + start_off);
    m.tiling = reinterpret_cast<int8_t*>(ds.group_buf + tiling_off);
  }
  CK(cudaMemcpy(ds.group_buf, host.data(), bytes, cudaMemcpyHostToDevice));
}

static void ensure_device(Plan& p) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (p.dev) {
    if (p.dev->device != dev) fail(TN_ERR_ARG, "plan was first used on another device");
    return;
  }
  auto* ds = new DeviceState;
  p.dev = ds;
  ds->device = dev;
  const size_t ab = std::max<size_t>(256, (size_t)p.arena_elems * sizeof(float2));
  if (cudaMalloc(&ds->arena, ab) != cudaSuccess) {
    cudaGetLastError();
    fail(TN_ERR_OOM, "arena allocation of " + std::to_string(ab) + " bytes failed");
  }
  const size_t lb = std::max<size_t>(16, p.leaf_data.size() * sizeof(float2));
  CK(cudaMalloc(&ds->leaf_data, lb));
  CK(cudaMemcpy(ds->leaf_data, p.leaf_data.data(), p.leaf_data.size() * sizeof(float2),
                cudaMemcpyHostToDevice));
  CK(cudaMalloc(&ds->leaf_desc, std::max<size_t>(1, p.leaves.size()) * sizeof(LeafDesc)));
  CK(cudaMemcpy(ds->leaf_desc, p.leaves.data(), p.leaves.size() * sizeof(LeafDesc),
                cudaMemcpyHostToDevice));
  CK(cudaMalloc(&ds->counter, sizeof(unsigned)));
  CK(cudaMalloc(&ds->err, sizeof(int32_t)));
  CK(cudaMemset(ds->err, 0, sizeof(int32_t)));
  CK(cudaEventCreateWithFlags(&ds->done, cudaEventDisableTiming));
  if (p.opts.precision == TN_PREC_FP16X3) {
    // leaves' maxima are constants of the plan; the steps' are recorded per chunk
    const size_t nn = p.leaves.size() + p.steps.size();
    CK(cudaMalloc(&ds->amax, sizeof(float) * std::max<size_t>(nn, 1)));
    CK(cudaMemset(ds->amax, 0, sizeof(float) * std::max<size_t>(nn, 1)));
    if (!p.leaf_amax.empty())
      CK(cudaMemcpy(ds->amax, p.leaf_amax.data(), sizeof(float) * p.leaf_amax.size(), cudaMemcpyHostToDevice));
  }
  // bounds of every operand inside the arena, checked once on the host
  const int64_t ae = p.arena_elems;
  auto in_arena = [&](int64_t off, int64_t size, int insts) {
    return off >= 0 && off + size * (int64_t)insts <= ae;
  };
  for (const LeafDesc& l : p.leaves)
    if (!in_arena(l.dst_off, (int64_t)1 << l.rank, 1 << __builtin_popcount(l.bmask)))
      fail(TN_ERR_PLAN, "internal: leaf outside the arena");
  for (const StepDesc& d : p.steps) {
    // every bit position must address inside the operand's own extent
    auto span_ok = [](const int8_t* pos, int n, int64_t elems) {
      for (int i = 0; i < n; ++i)
        if (pos[i] < 0 || ((int64_t)1 << pos[i]) >= elems) return false;
      return true;
    };
    const bool ok = in_arena(d.a_off, d.a_elems, 1) && in_arena(d.b_off, d.b_elems, 1) &&
                    in_arena(d.c_off, d.c_elems, 1) && span_ok(d.a_mpos, d.nm, d.a_elems) &&
                    span_ok(d.a_kpos, d.nk, d.a_elems) && span_ok(d.b_kpos, d.nk, d.b_elems) &&
                    span_ok(d.b_npos, d.nn, d.b_elems) && span_ok(d.c_mpos, d.nm, d.c_elems) &&
                    span_ok(d.c_npos, d.nn, d.c_elems) && span_ok(d.a_bpos, d.nb, d.a_elems) &&
                    span_ok(d.b_bpos, d.nb, d.b_elems) && span_ok(d.c_bpos, d.nb, d.c_elems) &&
                    ((int64_t)1 << (d.nm + d.nk + d.nb)) == d.a_elems &&
                    ((int64_t)1 << (d.nk + d.nn + d.nb)) == d.b_elems &&
                    ((int64_t)1 << (d.nm + d.nn + d.nb)) == d.c_elems;
    if (!ok) fail(TN_ERR_PLAN, "internal: step operand outside its extent");
    const int kid = pick_kernel(p.opts.precision, p.opts.complex_mult, d);
    ds->launches.push_back(make_launch(step_args(*ds, d, kid), kid, 64 - __builtin_clzll((uint64_t)d.a_elems) - 1, 1,
                                       d.c_elems, true, -1, (int64_t)256 << 20, 0, p.opts.sm_pairs ? -1 : 0));
  }
  int64_t ws = 16;
  for (const StepLaunch& L : ds->launches) ws = std::max(ws, L.ws_bytes);
  if (cudaMalloc(&ds->ws, (size_t)ws) != cudaSuccess) {
    cudaGetLastError();
    fail(TN_ERR_OOM, "workspace allocation of " + std::to_string(ws) + " bytes failed");
  }
  ds->ws_bytes = ws;
  ds->root_groups = std::min(1 << p.log2_batch, 64);
  CK(cudaMalloc(&ds->root_part, sizeof(double2) * (size_t)ds->root_groups << p.root.rank));
  if (!in_arena(p.root.off, (int64_t)1 << p.root.rank, 1 << __builtin_popcount(p.root.bmask)))
    fail(TN_ERR_PLAN, "internal: root outside the arena");
  build_groups(p, *ds);
  setup_hoisted(p, *ds);
}

void destroy_device_state(Plan* p) {
  if (!p || !p->dev) return;
  DeviceState* ds = p->dev;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(ds->device);
  if (ds->have_done) cudaEventSynchronize(ds->done);
  cudaFree(ds->arena);
  cudaFree(ds->leaf_data);
  cudaFree(ds->leaf_desc);
  cudaFree(ds->params);
  cudaFree(ds->counter);
  cudaFree(ds->err);
  cudaFree(ds->ws);
  cudaFree(ds->root_part);
  cudaFree(ds->amax);
  cudaFree(ds->group_buf);
  for (uint8_t* b : ds->own_imgs) cudaFree(b);
  if (ds->graph) cudaGraphExecDestroy(ds->graph);
  if (ds->done) cudaEventDestroy(ds->done);
  cudaSetDevice(cur);
  delete ds;
  p->dev = nullptr;
}

// The steps whose dependence flags satisfy `in_class`, in plan order; a group
// of independent small steps runs as its multi-step launches, then the rest of
// the group alone.
template <class Pred>
static void launch_class(Plan& p, cudaStream_t s, Pred in_class) {
  DeviceState& ds = *p.dev;
  for (size_t i = 0; i < p.steps.size(); ++i) {
    if (!in_class(p.steps[i].dep_flags)) continue;
    const int gi = ds.group_at.empty() ? -1 : ds.group_at[i];
    if (gi < 0) {
      launch_step(ds.launches[i], ds.ws, ds.err, s);
      continue;
    }
    const DeviceState::GroupRun& gr = ds.groups[gi];
    for (const auto& m : gr.multi) launch_simt_multi(m, s);
    for (int t : gr.singles) launch_step(ds.launches[t], ds.ws, ds.err, s);
    i = (size_t)gr.end - 1;
  }
}

static void run_chunk(Plan& p, cudaStream_t s) {
  DeviceState& ds = *p.dev;
  const int nl = (int)p.leaves.size();
  k_leaf_select<<<std::max(1, std::min(nl, 4096)), 128, 0, s>>>(ds.leaf_data, ds.leaf_desc, nl, ds.arena,
                                                                 ds.params, ds.counter);
  launch_class(p, s, [](int f) { return (f & 1) != 0; });   // slice-dependent steps
  const int64_t nout = (int64_t)1 << p.root.rank;
  const int blocks = (int)std::min<int64_t>((nout + 255) / 256, 4096);
  k_root_partial<<<dim3(blocks, ds.root_groups), 256, 0, s>>>(ds.arena, p.root, p.log2_batch, ds.root_groups,
                                                               ds.root_part, ds.params, ds.counter);
  k_root_finish<<<blocks, 256, 0, s>>>(ds.root_part, ds.root_groups, p.root.rank, ds.params, ds.counter);
  k_advance<<<1, 1, 0, s>>>(ds.counter);
}

// The steps of one dependence class (0: neither slice nor bitstring, 2:
// bitstring only), after a leaf select with the current chunk's parameters.
static void run_prologue(Plan& p, cudaStream_t s, int cls) {
  DeviceState& ds = *p.dev;
  bool any = false;
  for (const StepDesc& d : p.steps) any = any || d.dep_flags == cls;
  for (const StepLaunch& L : ds.launches) any = any || (L.bimg_own && L.bimg_cls == cls);
  if (!any) return;
  const int nl = (int)p.leaves.size();
  k_leaf_select<<<std::max(1, std::min(nl, 4096)), 128, 0, s>>>(ds.leaf_data, ds.leaf_desc, nl, ds.arena,
                                                                 ds.params, ds.counter);
  launch_class(p, s, [cls](int f) { return f == cls; });
  // the B' images of later steps whose B this class completes
  for (const StepLaunch& L : ds.launches) {
    if (!L.bimg_own || L.bimg_cls != cls) continue;
    TcArgs t = L.tc;
    t.bimg = L.bimg_own;
    t.err = ds.err;
    launch_prep_kid(t, L.kid, s);
  }
}

// Capture run_chunk once into a graph (on a private stream, thread-local
// capture mode).  Any failure leaves the plan on eager launches.
static void capture_chunk_graph(Plan& p) {
  DeviceState& ds = *p.dev;
  if (ds.graph || ds.graph_failed) return;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    ds.graph_failed = true;
    return;
  }
  cudaGraph_t graph = nullptr;
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    try {
      run_chunk(p, cs);
    } catch (const TnError&) {
      ok = false;
    }
    ok = (cudaStreamEndCapture(cs, &graph) == cudaSuccess) && ok;
  }
  if (ok) ok = cudaGraphInstantiate(&ds.graph, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (!ok) {
    cudaGetLastError();
    ds.graph = nullptr;
    ds.graph_failed = true;
  }
}

}  // namespace tnx

using namespace tnx;

#define API_BEGIN \
  try {           \
    clear_error();
#define API_END                        \
  return TN_OK;                        \
  }                                    \
  catch (const TnError& e) {           \
    set_error(e.msg);                  \
    return e.code;                     \
  }                                    \
  catch (const std::bad_alloc&) {      \
    set_error("host allocation failed"); \
    return TN_ERR_OOM;                 \
  }

extern "C" tn_status tn_contract_slices(tn_plan_t* h, uint64_t first, uint64_t count,
                                        const uint64_t* bitstrings, int32_t n_batches, double* out,
                                        void* stream) {
  API_BEGIN
  if (!h || !bitstrings || !out) fail(TN_ERR_ARG, "tn_contract_slices: NULL argument");
  Plan& p = h->plan;
  if (p.sticky != TN_OK) fail(p.sticky, p.sticky_msg);
  if (n_batches < 1) fail(TN_ERR_ARG, "n_batches must be >= 1");
  const int S = (int)p.sliced.size();
  const uint64_t total = S >= 64 ? ~0ULL : (1ULL << S);
  if (first > total || count > total - first) fail(TN_ERR_ARG, "slice range beyond 2^S");
  if (count == 0) return TN_OK;
  cudaStream_t s = (cudaStream_t)stream;
  ensure_device(p);
  DeviceState& ds = *p.dev;
  const int b = p.log2_batch;
  const uint64_t step = 1ULL << b;
  uint64_t open_mask = 0;
  for (int q : p.open_qubits) open_mask |= 1ULL << q;
  std::vector<ChunkParam> prm;
  for (int i = 0; i < n_batches; ++i)
    for (uint64_t base = (first >> b) << b; base < first + count; base += step) {
      ChunkParam c;
      c.slice_base = base;
      c.valid_lo = std::max(first, base);
      c.valid_hi = std::min(first + count, base + step);
      c.bitstring = bitstrings[i] & ~open_mask;
      c.out_index = i;
      c.out = out;
      prm.push_back(c);
    }
  if (ds.have_done) CK(cudaStreamWaitEvent(s, ds.done, 0));
  if (prm.size() > ds.params_cap) {
    if (ds.params) {
      CK(cudaStreamSynchronize(s));
      CK(cudaFree(ds.params));
      ds.params = nullptr;
    }
    ds.params_cap = std::max<size_t>(prm.size(), 1024);
    CK(cudaMalloc(&ds.params, ds.params_cap * sizeof(ChunkParam)));
  }
  CK(cudaMemcpyAsync(ds.params, prm.data(), prm.size() * sizeof(ChunkParam), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(ds.counter, 0, sizeof(unsigned), s));
  for (size_t c = 0; c < prm.size(); ++c) {
    if (c == 0 || prm[c].out_index != prm[c - 1].out_index) {   // first chunk of a batch
      if (!ds.pro0_done) {
        run_prologue(p, s, 0);
        ds.pro0_done = true;
      }
      if (!ds.pro2_valid || ds.pro2_bits != prm[c].bitstring) {
        run_prologue(p, s, 2);
        ds.pro2_valid = true;
        ds.pro2_bits = prm[c].bitstring;
      }
      CK(cudaGetLastError());
    }
    if (!ds.eager_done) {
      run_chunk(p, s);           // the first chunk runs eagerly (sets kernel attributes)
      CK(cudaGetLastError());
      ds.eager_done = true;
      capture_chunk_graph(p);
      continue;
    }
    if (ds.graph)
      CK(cudaGraphLaunch(ds.graph, s));
    else
      run_chunk(p, s);
    CK(cudaGetLastError());
  }
  CK(cudaEventRecord(ds.done, s));
  ds.have_done = true;
  API_END
}

extern "C" tn_status tn_plan_step_times(tn_plan_t* h, int32_t reps, double* ms_out, int32_t* kernel_out,
                                        void* stream) {
  API_BEGIN
  if (!h || !ms_out) fail(TN_ERR_ARG, "tn_plan_step_times: NULL argument");
  if (reps < 1) fail(TN_ERR_ARG, "tn_plan_step_times: reps must be >= 1");
  Plan& p = h->plan;
  if (!p.dev) fail(TN_ERR_ARG, "tn_plan_step_times: run tn_contract_slices first");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceState& ds = *p.dev;
  if (ds.have_done) CK(cudaStreamWaitEvent(s, ds.done, 0));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (size_t i = 0; i < p.steps.size(); ++i) {
    launch_step(ds.launches[i], ds.ws, ds.err, s);  // warm-up
    CK(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) launch_step(ds.launches[i], ds.ws, ds.err, s);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    ms_out[i] = (double)ms / reps;
    if (kernel_out) kernel_out[i] = ds.launches[i].kid;
  }
  CK(cudaGetLastError());
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ds.pro0_done = false;   // the arena was overwritten: prologues run again
  ds.pro2_valid = false;
  API_END
}

// Step d's launch with one kernel choice (as the autotuner builds its candidates).
static StepLaunch build_choice(const DeviceState& ds, const StepDesc& d, int kid, int tn_log, int epi, int bslots,
                               int pair) {
  return make_launch(step_args(ds, d, kid, tn_log), kid, 64 - __builtin_clzll((uint64_t)d.a_elems) - 1, 1,
                     d.c_elems, true, epi, (int64_t)256 << 20, bslots, pair);
}

// After the kernels of a plan changed: group runs, chunk graph and prologues anew.
static void kernels_changed(Plan& p, DeviceState& ds) {
  build_groups(p, ds);
  setup_hoisted(p, ds);
  if (ds.graph) {
    cudaGraphExecDestroy(ds.graph);
    ds.graph = nullptr;
  }
  ds.graph_failed = false;
  ds.eager_done = false;
  ds.pro0_done = false;   // the arena may have been overwritten: prologues run again
  ds.pro2_valid = false;
}

// Autotuner: for every step, time the candidate kernels in place (tensor-core
// tiles of 32, 64 or 128 complex columns in the TF32 / BF16X3 / FP16X3 modes,
// each with either write-back order, with the default or a deeper B' ring (4,
// 6 or 8 slots) and on one SM or an SM pair, and the three CUDA-core tilings
// where the step is small or the mode is FP32) and keep the fastest.  The
// chunk graph is captured again on the next call.
extern "C" tn_status tn_plan_autotune(tn_plan_t* h, int32_t reps, void* stream) {
  API_BEGIN
  if (!h) fail(TN_ERR_ARG, "tn_plan_autotune: NULL plan");
  if (reps < 1) fail(TN_ERR_ARG, "tn_plan_autotune: reps must be >= 1");
  Plan& p = h->plan;
  if (!p.dev) fail(TN_ERR_ARG, "tn_plan_autotune: run tn_contract_slices first");
  DeviceState& ds = *p.dev;
  cudaStream_t s = (cudaStream_t)stream;
  if (ds.have_done) CK(cudaStreamWaitEvent(s, ds.done, 0));
  CK(cudaStreamSynchronize(s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto time_launch = [&](StepLaunch& L) -> double {
    if (L.ws_bytes > ds.ws_bytes) {
      CK(cudaStreamSynchronize(s));
      CK(cudaFree(ds.ws));
      ds.ws = nullptr;
      ds.ws_bytes = 0;
      if (cudaMalloc(&ds.ws, (size_t)L.ws_bytes) != cudaSuccess) {
        cudaGetLastError();
        fail(TN_ERR_OOM, "autotune workspace allocation failed");
      }
      ds.ws_bytes = L.ws_bytes;
    }
    launch_step(L, ds.ws, ds.err, s);  // warm-up
    CK(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) launch_step(L, ds.ws, ds.err, s);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    return (double)ms / reps;
  };
  for (size_t i = 0; i < p.steps.size(); ++i) {
    const StepDesc& d = p.steps[i];
    auto build = [&](int kid, int tn_log, int epi, int bslots, int pair) {
      return build_choice(ds, d, kid, tn_log, epi, bslots, pair);
    };
    StepLaunch cur = ds.launches[i];
    cur.bimg_own = nullptr;   // timed like the candidates: B' images built with the launch
    double best = time_launch(cur);
    // kernel, tile width (log2 complex columns), write-back, B' slots, SM pairs
    std::vector<std::array<int, 5>> cands;
    const bool tc_mode = p.opts.precision != TN_PREC_FP32;
    const int tc_kid = tc_kernel(p.opts.precision, p.opts.complex_mult);
    if (tc_mode && d.nm >= 4)
      for (int tn_log : {7, 6, 5})
        if (tn_log <= std::max(3, d.nn))
          for (int epi : {0, 1})
            for (int bs : {0, 4, 6, 8})
              for (int pair : {1, 0})
                if (pair == 0 || p.opts.sm_pairs) cands.push_back({tc_kid, tn_log, epi, bs, pair});
    // CUDA-core tilings: FP32 mode, tiny steps, and low arithmetic intensity
    // (complex flops per byte moved), where a tile's fixed cost on the tensor
    // cores outweighs its few products
    const double flops = 8.0 * std::ldexp(1.0, d.nm + d.nk + d.nn + d.nb);
    const double bytes = 8.0 * (double)(d.a_elems + d.b_elems + d.c_elems);
    if (!tc_mode || best < 0.05 || flops / bytes < 48.0)
      for (int k : {K_SIMT_64x64, K_SIMT_128x16, K_SIMT_256x4}) cands.push_back({k, -1, 0, 0, 0});
    std::vector<std::array<int, 5>> seen;
    auto key = [](const StepLaunch& L) {
      return std::array<int, 5>{L.kid, L.g.tn, is_tc(L.kid) ? L.tc.epi_ok : 0, is_tc(L.kid) ? L.tc.nbs : 0,
                                is_tc(L.kid) ? L.tc.pair : 0};
    };
    seen.push_back(key(ds.launches[i]));
    for (auto [kid, tn_log, epi, bs, pair] : cands) {
      StepLaunch L;
      try {
        L = build(kid, tn_log, epi, bs, pair);
      } catch (const TnError&) {
        continue;   // this configuration does not fit: not a candidate
      }
      if (std::find(seen.begin(), seen.end(), key(L)) != seen.end()) continue;
      seen.push_back(key(L));
      const double t = time_launch(L);
      if (t < best * 0.97) {
        best = t;
        ds.launches[i] = L;
      }
    }
  }
  CK(cudaGetLastError());
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  kernels_changed(p, ds);
  API_END
}

extern "C" tn_status tn_plan_get_tuning(const tn_plan_t* h, int32_t* out, int32_t cap, int32_t* n_out) {
  API_BEGIN
  if (!h || !out || !n_out) fail(TN_ERR_ARG, "tn_plan_get_tuning: NULL argument");
  const Plan& p = h->plan;
  if (!p.dev) fail(TN_ERR_ARG, "tn_plan_get_tuning: run tn_contract_slices first");
  const int64_t need = (int64_t)p.steps.size() * TN_TUNING_INTS;
  if (cap < need) fail(TN_ERR_ARG, "tn_plan_get_tuning: cap below n_steps * TN_TUNING_INTS");
  for (size_t i = 0; i < p.steps.size(); ++i) {
    const StepLaunch& L = p.dev->launches[i];
    int32_t* o = out + i * TN_TUNING_INTS;
    const bool tc = is_tc(L.kid);
    o[0] = L.kid;
    o[1] = tc ? L.g.tn : -1;
    o[2] = tc ? L.tc.epi_ok : 0;
    o[3] = tc ? L.tc.nbs : 0;
    o[4] = tc ? L.tc.pair : 0;
  }
  *n_out = (int32_t)need;
  API_END
}

extern "C" tn_status tn_plan_set_tuning(tn_plan_t* h, const int32_t* in, int32_t n) {
  API_BEGIN
  if (!h || !in) fail(TN_ERR_ARG, "tn_plan_set_tuning: NULL argument");
  Plan& p = h->plan;
  if (!p.dev) fail(TN_ERR_ARG, "tn_plan_set_tuning: run tn_contract_slices first");
  if ((int64_t)n != (int64_t)p.steps.size() * TN_TUNING_INTS)
    fail(TN_ERR_ARG, "tn_plan_set_tuning: n is not n_steps * TN_TUNING_INTS");
  DeviceState& ds = *p.dev;
  std::vector<StepLaunch> next(p.steps.size());
  int64_t ws = ds.ws_bytes;
  for (size_t i = 0; i < p.steps.size(); ++i) {
    const int32_t* c = in + i * TN_TUNING_INTS;
    const int kid = c[0];
    const bool simt = kid == K_SIMT_64x64 || kid == K_SIMT_128x16 || kid == K_SIMT_256x4;
    if (!simt && !is_tc(kid)) fail(TN_ERR_ARG, "tn_plan_set_tuning: unknown kernel id");
    if (is_tc(kid) && (p.opts.precision == TN_PREC_FP32 || kid != tc_kernel(p.opts.precision, p.opts.complex_mult)))
      fail(TN_ERR_ARG, "tn_plan_set_tuning: tensor-core kernel of another precision or product");
    if (c[2] < 0 || c[2] > 1 || c[3] < 0 || c[3] > TC_MAX_B || c[4] < 0 || c[4] > 1 || c[1] < -1 || c[1] > 7)
      fail(TN_ERR_ARG, "tn_plan_set_tuning: choice out of range");
    try {
      next[i] = simt ? build_choice(ds, p.steps[i], kid, -1, 0, 0, 0)
                     : build_choice(ds, p.steps[i], kid, c[1], c[2], c[3], c[4] && p.opts.sm_pairs ? 1 : 0);
    } catch (const TnError& e) {
      fail(TN_ERR_ARG, std::string("tn_plan_set_tuning: step ") + std::to_string(i) + ": " + e.msg);
    }
    ws = std::max(ws, next[i].ws_bytes);
  }
  if (ws > ds.ws_bytes) {   // a larger workspace (synchronises the device through cudaFree)
    CK(cudaFree(ds.ws));
    ds.ws = nullptr;
    ds.ws_bytes = 0;
    if (cudaMalloc(&ds.ws, (size_t)ws) != cudaSuccess) {
      cudaGetLastError();
      fail(TN_ERR_OOM, "tn_plan_set_tuning: workspace allocation failed");
    }
    ds.ws_bytes = ws;
  }
  ds.launches.swap(next);
  kernels_changed(p, ds);
  API_END
}

// Time one chunk of every candidate (seed and memory weight per candidate, the
// rest from *opts) after an untimed warm-up chunk, and keep the plan whose
// estimate for all 2^S slices is smallest.
static void select_among(const tn_network_t* net, const tn_plan_opts* opts, int32_t n_candidates,
                         const uint64_t* seeds, const double* weights, uint64_t bitstring, void* stream,
                         tn_plan_t** out, double* cand_seconds) {
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  tn_plan_t* best = nullptr;
  double best_t = 0.0;
  double* amps = nullptr;
  size_t amps_bytes = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int i = 0; i < n_candidates; ++i) {
    if (cand_seconds) cand_seconds[i] = -1.0;
    tn_plan_opts o = *opts;
    o.seed = seeds[i];
    o.mem_weight = weights[i];
    tn_plan_t* h = nullptr;
    if (tn_plan(net, &o, &h) != TN_OK || !h) continue;
    Plan& p = h->plan;
    const uint64_t chunk = 1ULL << p.log2_batch;
    const size_t need = sizeof(double) * 2 * ((size_t)1 << p.root.rank);
    if (need > amps_bytes) {
      if (amps) CK(cudaFree(amps));
      amps = nullptr;
      CK(cudaMalloc(&amps, need));
      amps_bytes = need;
    }
    double est = -1.0;
    // warm-up (device state, prologues, graph capture), then the fastest of
    // three timed chunks
    if (tn_contract_slices(h, 0, chunk, &bitstring, 1, amps, s) == TN_OK) {
      float best_ms = -1.f;
      tn_status st = TN_OK;
      for (int r = 0; r < 3 && st == TN_OK; ++r) {
        CK(cudaEventRecord(e0, s));
        st = tn_contract_slices(h, 0, chunk, &bitstring, 1, amps, s);
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (best_ms < 0.f || ms < best_ms) best_ms = ms;
      }
      if (st == TN_OK && tn_plan_sync(h, s) == TN_OK)
        est = (double)best_ms / 1e3 * std::ldexp(1.0, (int)p.sliced.size() - p.log2_batch);
    }
    CK(cudaStreamSynchronize(s));
    destroy_device_state(&p);
    cudaGetLastError();
    clear_error();
    if (cand_seconds) cand_seconds[i] = est;
    if (est >= 0.0 && (!best || est < best_t)) {
      if (best) tn_plan_destroy(best);
      best = h;
      best_t = est;
    } else {
      tn_plan_destroy(h);
    }
  }
  if (amps) cudaFree(amps);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!best) fail(TN_ERR_PLAN, "plan selection: no candidate plan could be built and run");
  best->plan.sticky = TN_OK;
  *out = best;
}

extern "C" tn_status tn_plan_select(const tn_network_t* net, const tn_plan_opts* opts, int32_t n_candidates,
                                    uint64_t bitstring, void* stream, tn_plan_t** out, double* cand_seconds) {
  API_BEGIN
  if (!net || !opts || !out) fail(TN_ERR_ARG, "tn_plan_select: NULL argument");
  if (n_candidates < 1 || n_candidates > 1024) fail(TN_ERR_ARG, "tn_plan_select: n_candidates must be in [1, 1024]");
  const double w0 = opts->mem_weight > 0.0 ? opts->mem_weight : 32.0;
  const double wmul[3] = {1.0, 0.25, 4.0};
  std::vector<uint64_t> seeds(n_candidates);
  std::vector<double> weights(n_candidates);
  for (int i = 0; i < n_candidates; ++i) {
    seeds[i] = opts->seed + (uint64_t)i;
    weights[i] = w0 * wmul[i % 3];
  }
  select_among(net, opts, n_candidates, seeds.data(), weights.data(), bitstring, stream, out, cand_seconds);
  API_END
}

extern "C" tn_status tn_plan_select_list(const tn_network_t* net, const tn_plan_opts* opts, int32_t n_candidates,
                                         const uint64_t* seeds, const double* mem_weights, uint64_t bitstring,
                                         void* stream, tn_plan_t** out, double* cand_seconds) {
  API_BEGIN
  if (!net || !opts || !out || !seeds || !mem_weights) fail(TN_ERR_ARG, "tn_plan_select_list: NULL argument");
  if (n_candidates < 1 || n_candidates > 1024)
    fail(TN_ERR_ARG, "tn_plan_select_list: n_candidates must be in [1, 1024]");
  for (int i = 0; i < n_candidates; ++i)
    if (!(mem_weights[i] <= 0.0 || (mem_weights[i] >= 1e-6 && mem_weights[i] <= 1e9)))
      fail(TN_ERR_ARG, "tn_plan_select_list: mem_weight must be <= 0 (default) or in [1e-6, 1e9]");
  select_among(net, opts, n_candidates, seeds, mem_weights, bitstring, stream, out, cand_seconds);
  API_END
}

// Kernels launch_class launches for the steps of a class (memsets not counted).
template <class Pred>
static int class_launches(const Plan& p, Pred in_class) {
  int n = 0;
  auto kernels_of = [&](int i) {
    const StepLaunch& L = p.dev->launches[i];
    return is_tc(L.kid) ? (L.tc.n_split > 1 ? 3 : 2) - (L.bimg_own ? 1 : 0) : 1;
  };
  for (size_t i = 0; i < p.steps.size(); ++i) {
    if (!in_class(p.steps[i].dep_flags)) continue;
    const int gi = p.dev->group_at.empty() ? -1 : p.dev->group_at[i];
    if (gi < 0) {
      n += kernels_of((int)i);
      continue;
    }
    const auto& gr = p.dev->groups[gi];
    n += (int)gr.multi.size();
    for (int t : gr.singles) n += kernels_of(t);
    i = (size_t)gr.end - 1;
  }
  return n;
}

extern "C" tn_status tn_plan_chunk_launches(const tn_plan_t* h, int32_t* launches) {
  API_BEGIN
  if (!h || !launches) fail(TN_ERR_ARG, "tn_plan_chunk_launches: NULL argument");
  const Plan& p = h->plan;
  if (!p.dev) fail(TN_ERR_ARG, "tn_plan_chunk_launches: call after the first tn_contract_slices");
  *launches = 4 + class_launches(p, [](int f) { return (f & 1) != 0; });
  API_END
}

extern "C" tn_status tn_plan_batch_launches(const tn_plan_t* h, int32_t* launches) {
  API_BEGIN
  if (!h || !launches) fail(TN_ERR_ARG, "tn_plan_batch_launches: NULL argument");
  const Plan& p = h->plan;
  if (!p.dev) fail(TN_ERR_ARG, "tn_plan_batch_launches: call after the first tn_contract_slices");
  int n = class_launches(p, [](int f) { return f == 2; });
  for (const StepLaunch& L : p.dev->launches) n += (L.bimg_own && L.bimg_cls == 2) ? 1 : 0;   // B' images
  *launches = n > 0 ? n + 1 : 0;   // + the leaf select ahead of them
  API_END
}

extern "C" tn_status tn_plan_sync(tn_plan_t* h, void* stream) {
  API_BEGIN
  if (!h) fail(TN_ERR_ARG, "tn_plan_sync: NULL plan");
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  if (h->plan.dev && h->plan.sticky == TN_OK) {
    int32_t e = 0;
    CK(cudaMemcpy(&e, h->plan.dev->err, sizeof(e), cudaMemcpyDeviceToHost));
    if (e != 0) {
      h->plan.sticky = e;
      h->plan.sticky_msg = "a device kernel reported error " + std::to_string(e) +
                           " (bounded wait expired or device check failed)";
    }
  }
  if (h->plan.sticky != TN_OK) fail(h->plan.sticky, h->plan.sticky_msg);
  API_END
}

extern "C" void tn_plan_destroy(tn_plan_t* h) {
  if (!h) return;
  destroy_device_state(&h->plan);
  delete h;
}

// Per-device scratch of the calls that have no plan: the XEB sum, the error
// word and the B' workspace of tn_contract_pair.
// FP16X3 calls without a plan: the maxima of A and B by one reduction pass each
static void operand_maxima(const float2* a, int64_t na, const float2* b, int64_t nb, float* amax, cudaStream_t s) {
  CK(cudaMemsetAsync(amax, 0, 2 * sizeof(float), s));
  const int ga = (int)std::min<int64_t>((na + 255) / 256, (int64_t)sm_count() * 8);
  const int gb = (int)std::min<int64_t>((nb + 255) / 256, (int64_t)sm_count() * 8);
  k_amax<<<std::max(ga, 1), 256, 0, s>>>(a, na, amax);
  k_amax<<<std::max(gb, 1), 256, 0, s>>>(b, nb, amax + 1);
}

struct Scratch {
  double* xeb = nullptr;
  int32_t* err = nullptr;
  float* amax = nullptr;   // FP16X3 operand maxima of the last call (A, B)
  unsigned long long* first = nullptr;   // frugal sampling: first accepted draw per sample
  int64_t first_cap = 0;
  int32_t* bad = nullptr;
  uint8_t* ws = nullptr;
  int64_t ws_bytes = 0;
};
static std::mutex g_scratch_mu;
static std::unordered_map<int, Scratch> g_scratch;   // per device
static Scratch& scratch_for_device() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  Scratch& s = g_scratch[dev];
  if (!s.xeb) {
    CK(cudaMalloc(&s.xeb, sizeof(double)));
    CK(cudaMalloc(&s.err, sizeof(int32_t)));
    CK(cudaMemset(s.err, 0, sizeof(int32_t)));
    CK(cudaMalloc(&s.amax, 2 * sizeof(float)));
    CK(cudaMalloc(&s.bad, sizeof(int32_t)));
  }
  return s;
}

extern "C" tn_status tn_xeb(const double* amps, int64_t count, int32_t n_qubits, double* xeb_out,
                            void* stream) {
  API_BEGIN
  if (!amps || !xeb_out) fail(TN_ERR_ARG, "tn_xeb: NULL argument");
  if (count < 1) fail(TN_ERR_ARG, "tn_xeb: count must be >= 1");
  if (n_qubits < 0 || n_qubits > 1023) fail(TN_ERR_ARG, "tn_xeb: n_qubits out of range");
  double* scratch = scratch_for_device().xeb;
  cudaStream_t s = (cudaStream_t)stream;
  k_xeb_sum<<<1, 1024, 0, s>>>(reinterpret_cast<const double2*>(amps), count, scratch);
  CK(cudaGetLastError());
  double sum = 0;
  CK(cudaMemcpyAsync(&sum, scratch, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *xeb_out = std::ldexp(sum / (double)count, n_qubits) - 1.0;
  API_END
}

extern "C" tn_status tn_frugal_sample(const double* amps, int64_t count, int32_t n_qubits, double m_bound,
                                     const int64_t* candidates, const double* uniforms, int64_t n_draws,
                                     int64_t n_samples, int64_t* first_out, void* stream) {
  API_BEGIN
  if (!amps || !candidates || !uniforms || !first_out) fail(TN_ERR_ARG, "tn_frugal_sample: NULL argument");
  if (count < 1 || n_draws < 1 || n_samples < 1) fail(TN_ERR_ARG, "tn_frugal_sample: empty batch, draws or samples");
  if (n_qubits < 0 || n_qubits > 1000) fail(TN_ERR_ARG, "tn_frugal_sample: n_qubits out of range");
  if (!(m_bound > 0.0) || !std::isfinite(m_bound)) fail(TN_ERR_ARG, "tn_frugal_sample: m_bound must be positive");
  if (n_draws > ((int64_t)1 << 40) / n_samples) fail(TN_ERR_ARG, "tn_frugal_sample: too many draws");
  Scratch& sc = scratch_for_device();
  cudaStream_t s = (cudaStream_t)stream;
  if (n_samples > sc.first_cap) {
    CK(cudaStreamSynchronize(s));
    if (sc.first) CK(cudaFree(sc.first));
    sc.first = nullptr;
    CK(cudaMalloc(&sc.first, sizeof(unsigned long long) * (size_t)n_samples));
    sc.first_cap = n_samples;
  }
  CK(cudaMemsetAsync(sc.first, 0xff, sizeof(unsigned long long) * (size_t)n_samples, s));
  CK(cudaMemsetAsync(sc.bad, 0, sizeof(int32_t), s));
  const int64_t total = n_draws * n_samples;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sm_count() * 16);
  k_frugal<<<blocks, 256, 0, s>>>(reinterpret_cast<const double2*>(amps), count, n_qubits, m_bound, candidates,
                                  uniforms, n_draws, n_samples, sc.first, sc.bad);
  CK(cudaGetLastError());
  std::vector<unsigned long long> f((size_t)n_samples);
  int32_t bad = 0;
  CK(cudaMemcpyAsync(f.data(), sc.first, sizeof(unsigned long long) * f.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&bad, sc.bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (bad) fail(TN_ERR_ARG, "tn_frugal_sample: a candidate index is outside [0, count)");
  for (int64_t i = 0; i < n_samples; ++i) first_out[i] = f[i] == ~0ULL ? -1 : (int64_t)f[i];
  API_END
}

extern "C" tn_status tn_permute(const float* in, float* out, int32_t rank, const int32_t* perm,
                                int64_t batch, void* stream) {
  API_BEGIN
  if (!in || !out || (!perm && rank > 0)) fail(TN_ERR_ARG, "tn_permute: NULL argument");
  if (rank < 0 || rank > 34) fail(TN_ERR_ARG, "tn_permute: rank must be in [0, 34]");
  if (batch < 0) fail(TN_ERR_ARG, "tn_permute: negative batch");
  PermArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  std::vector<char> seen(rank, 0);
  for (int p = 0; p < rank; ++p) {
    if (perm[p] < 0 || perm[p] >= rank || seen[perm[p]]) fail(TN_ERR_ARG, "tn_permute: not a permutation");
    seen[perm[p]] = 1;
    pa.src_pos[p] = (int8_t)perm[p];
  }
  const int64_t total = batch << rank;
  if (total == 0) return TN_OK;
  if (rank < 10) {
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 64);
    k_permute_gather<<<blocks, 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const float2*>(in),
                                                               reinterpret_cast<float2*>(out), rank, pa, total);
  } else {
    // tile bits: input positions 0..4 and the inputs of output positions 0..4
    std::vector<int> out_of_in(rank);
    for (int p = 0; p < rank; ++p) out_of_in[perm[p]] = p;
    std::vector<char> in_tile(rank, 0);
    for (int i = 0; i < 5; ++i) in_tile[i] = 1;
    for (int p = 0; p < 5; ++p) in_tile[perm[p]] = 1;
    // widen to 10 tile bits: alternately the next input bit and the source of
    // the next output bit (longer contiguous runs on both sides)
    {
      int nt = 0;
      for (int i = 0; i < rank; ++i) nt += in_tile[i];
      int ni = 5, no = 5;
      while (nt < 10 && (ni < rank || no < rank)) {
        if (ni < rank && !in_tile[ni] && nt < 10) {
          in_tile[ni] = 1;
          ++nt;
        }
        ++ni;
        if (no < rank && !in_tile[perm[no]] && nt < 10) {
          in_tile[perm[no]] = 1;
          ++nt;
        }
        ++no;
      }
    }
    pa.nt = 0;
    pa.nr = 0;
    for (int i = 0; i < rank; ++i) {
      if (in_tile[i]) {
        pa.t_in[pa.nt] = (int8_t)i;
        pa.t_out[pa.nt] = (int8_t)out_of_in[i];
        ++pa.nt;
      } else {
        pa.r_in[pa.nr] = (int8_t)i;
        pa.r_out[pa.nr] = (int8_t)out_of_in[i];
        ++pa.nr;
      }
    }
    std::vector<int> ord(pa.nt);
    for (int q = 0; q < pa.nt; ++q) ord[q] = q;
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return pa.t_out[x] < pa.t_out[y]; });
    for (int q = 0; q < pa.nt; ++q) pa.t_out_order[q] = ord[q];
    const int64_t tiles = (int64_t)1 << pa.nr;
    const int blocks = (int)std::min<int64_t>(tiles * batch, (int64_t)sm_count() * 8);
    k_permute_tiled<<<blocks, 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const float2*>(in),
                                                              reinterpret_cast<float2*>(out), rank, pa, tiles,
                                                              batch);
  }
  CK(cudaGetLastError());
  API_END
}

extern "C" tn_status tn_contract_pair(const float* a, const int32_t* aw, int32_t ar, const float* b,
                                      const int32_t* bw, int32_t br, float* c, const int32_t* cw,
                                      int32_t cr, int64_t batch, int32_t precision, int32_t cmult,
                                      void* stream) {
  API_BEGIN
  if (!a || !b || !c || (ar && !aw) || (br && !bw) || (cr && !cw)) fail(TN_ERR_ARG, "tn_contract_pair: NULL argument");
  if (ar < 0 || br < 0 || cr < 0 || ar > 34 || br > 34 || cr > 34) fail(TN_ERR_ARG, "tn_contract_pair: rank out of range");
  if (batch < 1 || batch > 65535) fail(TN_ERR_ARG, "tn_contract_pair: batch must be in [1, 65535]");
  if (precision < TN_PREC_FP32 || precision > TN_PREC_FP16X3) fail(TN_ERR_ARG, "unknown precision");
  if (cmult != 3 && cmult != 4) fail(TN_ERR_ARG, "complex_mult must be 3 or 4");
  if (cmult == 3 && precision == TN_PREC_FP32)
    fail(TN_ERR_UNSUPPORTED, "the FP32 CUDA-core path forms 4M products only; 3M needs TF32 or BF16X3");
  std::vector<int> A(aw, aw + ar), B(bw, bw + br), Cw(cw, cw + cr);
  auto has = [](const std::vector<int>& v, int w) { return std::find(v.begin(), v.end(), w) != v.end(); };
  for (size_t i = 0; i < A.size(); ++i)
    for (size_t j = i + 1; j < A.size(); ++j)
      if (A[i] == A[j]) fail(TN_ERR_ARG, "repeated wire in a_wires");
  for (size_t i = 0; i < B.size(); ++i)
    for (size_t j = i + 1; j < B.size(); ++j)
      if (B[i] == B[j]) fail(TN_ERR_ARG, "repeated wire in b_wires");
  StepDesc d;
  std::memset(&d, 0, sizeof(d));
  std::vector<int> mw, kw, nw;
  for (int w : A) (has(B, w) ? kw : mw).push_back(w);
  for (int w : B)
    if (!has(A, w)) nw.push_back(w);
  if (mw.size() + nw.size() != Cw.size()) fail(TN_ERR_ARG, "c_wires must be the uncontracted wires");
  for (int w : mw)
    if (!has(Cw, w)) fail(TN_ERR_ARG, "c_wires misses a wire of A");
  for (int w : nw)
    if (!has(Cw, w)) fail(TN_ERR_ARG, "c_wires misses a wire of B");
  auto pos = [](const std::vector<int>& v, int w) { return (int)(std::find(v.begin(), v.end(), w) - v.begin()); };
  d.nm = (int)mw.size();
  d.nk = (int)kw.size();
  d.nn = (int)nw.size();
  for (int i = 0; i < d.nm; ++i) {
    d.a_mpos[i] = (int8_t)pos(A, mw[i]);
    d.c_mpos[i] = (int8_t)pos(Cw, mw[i]);
  }
  for (int j = 0; j < d.nk; ++j) {
    d.a_kpos[j] = (int8_t)pos(A, kw[j]);
    d.b_kpos[j] = (int8_t)pos(B, kw[j]);
  }
  for (int i = 0; i < d.nn; ++i) {
    d.b_npos[i] = (int8_t)pos(B, nw[i]);
    d.c_npos[i] = (int8_t)pos(Cw, nw[i]);
  }
  d.a_elems = (int64_t)1 << ar;
  d.b_elems = (int64_t)1 << br;
  d.c_elems = (int64_t)1 << cr;
  d.nb = 0;
  const int kid = pick_kernel(precision, cmult, d);
  GemmArgs g = make_args(d, kid, reinterpret_cast<const float2*>(a), reinterpret_cast<const float2*>(b),
                         reinterpret_cast<float2*>(c), (int32_t)batch, d.a_elems, d.b_elems, d.c_elems);
  Scratch& sc = scratch_for_device();
  if (precision == TN_PREC_FP16X3 && is_tc(kid)) {   // operand maxima for the FP16 scaling (one extra read)
    operand_maxima(reinterpret_cast<const float2*>(a), batch << ar, reinterpret_cast<const float2*>(b),
                   batch << br, sc.amax, (cudaStream_t)stream);
    g.amax_a = sc.amax;
    g.amax_b = sc.amax + 1;
  }
  StepLaunch L = make_launch(g, kid, ar, batch, batch * d.c_elems, true);
  if (L.ws_bytes > sc.ws_bytes) {
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    if (sc.ws) CK(cudaFree(sc.ws));
    sc.ws = nullptr;
    CK(cudaMalloc(&sc.ws, (size_t)L.ws_bytes));
    sc.ws_bytes = L.ws_bytes;
  }
  launch_step(L, sc.ws, sc.err, (cudaStream_t)stream);
  CK(cudaGetLastError());
  API_END
}

extern "C" tn_status tn_selftest_bounded_wait(int32_t wait_ms, int32_t* device_status, void* stream) {
  API_BEGIN
  if (!device_status) fail(TN_ERR_ARG, "tn_selftest_bounded_wait: NULL argument");
  if (wait_ms < 1 || wait_ms > 5000) fail(TN_ERR_ARG, "tn_selftest_bounded_wait: wait_ms must be in [1, 5000]");
  Scratch& sc = scratch_for_device();
  cudaStream_t s = (cudaStream_t)stream;
  k_selftest_wait<<<1, 32, 0, s>>>(sc.err, (uint64_t)wait_ms * 1000000ull);
  CK(cudaGetLastError());
  int32_t e = 0;
  CK(cudaMemcpyAsync(&e, sc.err, sizeof(e), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *device_status = e;   // the word stays set until tn_device_sync reads it
  API_END
}

// ---------------------------------------------------------------- no-allocation variant
// Some callers cannot call cudaMalloc at all: code running while a CUDA graph
// is being captured, allocation-free real-time or embedded hosts, and programs
// whose memory pool is owned by someone else.  tn_contract_pair_noalloc serves
// them with the same kernels as tn_contract_pair, taking its scratch (the
// device error word and the B' images of the tensor-core kernels) from this
// file-scope device array instead of allocating it.  Every GPU that loads the
// library holds the array until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;   // 32 MiB
constexpr size_t kNoAllocErrBytes = 256;                     // error word, then the B' images
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static std::unordered_map<int, void*> g_noalloc_addr;   // per device, found once with that device current

static void* noalloc_scratch_address() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  auto it = g_noalloc_addr.find(dev);
  if (it != g_noalloc_addr.end()) return it->second;
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    fail(TN_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array: ") + cudaGetErrorString(e));
  g_noalloc_addr[dev] = p;
  return p;
}

extern "C" tn_status tn_contract_pair_noalloc(const float* a, const int32_t* aw, int32_t ar, const float* b,
                                              const int32_t* bw, int32_t br, float* c, const int32_t* cw,
                                              int32_t cr, int64_t batch, int32_t precision, int32_t cmult,
                                              void* stream) {
  API_BEGIN
  if (!a || !b || !c || (ar && !aw) || (br && !bw) || (cr && !cw))
    fail(TN_ERR_ARG, "tn_contract_pair_noalloc: NULL argument");
  if (ar < 0 || br < 0 || cr < 0 || ar > 34 || br > 34 || cr > 34)
    fail(TN_ERR_ARG, "tn_contract_pair_noalloc: rank out of range");
  if (batch < 1 || batch > 65535) fail(TN_ERR_ARG, "tn_contract_pair_noalloc: batch must be in [1, 65535]");
  if (precision < TN_PREC_FP32 || precision > TN_PREC_FP16X3) fail(TN_ERR_ARG, "unknown precision");
  if (cmult != 3 && cmult != 4) fail(TN_ERR_ARG, "complex_mult must be 3 or 4");
  if (cmult == 3 && precision == TN_PREC_FP32)
    fail(TN_ERR_UNSUPPORTED, "the FP32 CUDA-core path forms 4M products only; 3M needs TF32 or BF16X3");
  std::vector<int> A(aw, aw + ar), B(bw, bw + br), Cw(cw, cw + cr);
  auto has = [](const std::vector<int>& v, int w) { return std::find(v.begin(), v.end(), w) != v.end(); };
  auto dup = [](const std::vector<int>& v) {
    for (size_t i = 0; i < v.size(); ++i)
      for (size_t j = i + 1; j < v.size(); ++j)
        if (v[i] == v[j]) return true;
    return false;
  };
  if (dup(A) || dup(B) || dup(Cw)) fail(TN_ERR_ARG, "repeated wire in a wire list");
  StepDesc d;
  std::memset(&d, 0, sizeof(d));
  std::vector<int> mw, kw, nw;
  for (int w : A) (has(B, w) ? kw : mw).push_back(w);
  for (int w : B)
    if (!has(A, w)) nw.push_back(w);
  if (mw.size() + nw.size() != Cw.size()) fail(TN_ERR_ARG, "c_wires must be the uncontracted wires");
  for (int w : mw)
    if (!has(Cw, w)) fail(TN_ERR_ARG, "c_wires misses a wire of A");
  for (int w : nw)
    if (!has(Cw, w)) fail(TN_ERR_ARG, "c_wires misses a wire of B");
  auto pos = [](const std::vector<int>& v, int w) { return (int)(std::find(v.begin(), v.end(), w) - v.begin()); };
  d.nm = (int)mw.size();
  d.nk = (int)kw.size();
  d.nn = (int)nw.size();
  for (int i = 0; i < d.nm; ++i) {
    d.a_mpos[i] = (int8_t)pos(A, mw[i]);
    d.c_mpos[i] = (int8_t)pos(Cw, mw[i]);
  }
  for (int j = 0; j < d.nk; ++j) {
    d.a_kpos[j] = (int8_t)pos(A, kw[j]);
    d.b_kpos[j] = (int8_t)pos(B, kw[j]);
  }
  for (int i = 0; i < d.nn; ++i) {
    d.b_npos[i] = (int8_t)pos(B, nw[i]);
    d.c_npos[i] = (int8_t)pos(Cw, nw[i]);
  }
  d.a_elems = (int64_t)1 << ar;
  d.b_elems = (int64_t)1 << br;
  d.c_elems = (int64_t)1 << cr;
  const int kid = pick_kernel(precision, cmult, d);
  GemmArgs g = make_args(d, kid, reinterpret_cast<const float2*>(a), reinterpret_cast<const float2*>(b),
                         reinterpret_cast<float2*>(c), (int32_t)batch, d.a_elems, d.b_elems, d.c_elems);
  const int64_t cap = (int64_t)(kNoAllocScratchBytes - kNoAllocErrBytes);
  uint8_t* base = static_cast<uint8_t*>(noalloc_scratch_address());
  int32_t* err = reinterpret_cast<int32_t*>(base);
  float* amax = reinterpret_cast<float*>(base + 16);   // FP16X3 operand maxima, inside the header
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == TN_PREC_FP16X3 && is_tc(kid)) {
    g.amax_a = amax;
    g.amax_b = amax + 1;
  }
  // split-K as tn_contract_pair chooses it, as long as the partial sums fit
  // beside the B' images; otherwise one pass over k
  StepLaunch L = make_launch(g, kid, ar, batch, batch * d.c_elems, true, -1, cap);
  if (L.ws_bytes > cap) L = make_launch(g, kid, ar, batch);
  if (L.ws_bytes > cap)
    fail(TN_ERR_ARG, "tn_contract_pair_noalloc: this contraction needs " + std::to_string(L.ws_bytes) +
                         " bytes of scratch; the static array holds " + std::to_string(cap));
  // the error word is zero when the library loads and is cleared by
  // tn_device_sync; kernels only ever set it, so it is not cleared here
  if (g.amax_a)
    operand_maxima(reinterpret_cast<const float2*>(a), batch << ar, reinterpret_cast<const float2*>(b),
                   batch << br, amax, s);
  launch_step(L, base + kNoAllocErrBytes, err, s);
  CK(cudaGetLastError());
  API_END
}

// ---------------------------------------------------------------- device error word
// Calls without a plan (tn_contract_pair, tn_contract_pair_noalloc,
// tn_selftest_bounded_wait) leave device-side errors in a per-device word: the
// scratch area's word, and the first word of the static array of the
// no-allocation entry point.  This reads both, clears what was set, and
// allocates nothing: a word that was never created cannot hold an error.
extern "C" tn_status tn_device_sync(void* stream) {
  API_BEGIN
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  int32_t* words[2] = {nullptr, nullptr};
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    auto it = g_scratch.find(dev);
    if (it != g_scratch.end()) words[0] = it->second.err;
  }
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    auto it = g_noalloc_addr.find(dev);
    if (it != g_noalloc_addr.end()) words[1] = static_cast<int32_t*>(it->second);
  }
  int32_t val[2] = {0, 0};
  for (int i = 0; i < 2; ++i)
    if (words[i]) CK(cudaMemcpyAsync(&val[i], words[i], sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int32_t e = 0;
  for (int i = 0; i < 2; ++i)
    if (val[i] != 0) {
      CK(cudaMemsetAsync(words[i], 0, sizeof(int32_t), s));
      if (e == 0) e = val[i];
    }
  if (e != 0) {
    CK(cudaStreamSynchronize(s));
    const tn_status code = (e == TN_ERR_TIMEOUT || e == TN_ERR_DEVICE || e == TN_ERR_ARG) ? e : TN_ERR_DEVICE;
    fail(code, "a device kernel of a call without a plan reported error " + std::to_string(e) +
                   (e == TN_ERR_TIMEOUT ? " (a bounded wait expired; its result is incomplete)" : ""));
  }
  API_END
}
