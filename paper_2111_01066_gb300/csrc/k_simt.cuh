// Complex GEMM on the CUDA cores (complex64, FP32 FMA): the plain FP32 path.
// Operands are gathered straight from their tensors' storage order, so the
// index permutation of SI Eq. (2) is folded into the loads (the paper's fused
// permutation-multiplication, SI figure S7a): each tile covers the lowest
// memory positions of its operand, so the gathers read contiguous runs.
#pragma once
#include "kernels_common.cuh"

namespace tnx {

// Shared memory of one tile of a tiling.
template <int TM, int TN, int TK>
struct SimtSmem {
  float2 As[TK][TM];
  float2 Bs[TK][TN];
  int64_t offCm[TM];
  int64_t offCn[TN];
};

// One (m tile bx, n tile by) of a GEMM for instances bz, bz + gz, ... (the
// body of both kernels below; every thread of the block calls it).
template <int TM, int TN, int TK, int RM, int RN>
__device__ __forceinline__ void simt_tile(const GemmArgs& g, int bx, int by, int bz, int gz,
                                          SimtSmem<TM, TN, TK>& sm) {
  constexpr int NTX = TM / RM, NTY = TN / RN, NT = NTX * NTY;
  constexpr int AE = (TM * TK + NT - 1) / NT;
  constexpr int BE = (TK * TN + NT - 1) / NT;
  auto& As = sm.As;
  auto& Bs = sm.Bs;
  auto& offCm = sm.offCm;
  auto& offCn = sm.offCn;
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;
  const int TMv = 1 << g.tm, TKv = 1 << g.tk, TNv = 1 << g.tn;

  for (int i = tid; i < TK * TM; i += NT) (&As[0][0])[i] = make_float2(0.f, 0.f);
  for (int i = tid; i < TK * TN; i += NT) (&Bs[0][0])[i] = make_float2(0.f, 0.f);
  for (int r = tid; r < TM; r += NT) offCm[r] = r < TMv ? deposit_hi((uint64_t)r, g.c_mpos, 0, g.tm) : 0;
  for (int c = tid; c < TN; c += NT) offCn[c] = c < TNv ? deposit_hi((uint64_t)c, g.c_npos, 0, g.tn) : 0;

  // Each thread's share of a tile, decoded once: element e of the tile has its
  // bits assigned to tile bits in ascending memory position, so consecutive e
  // (consecutive threads) read consecutive addresses.
  int a_sm[AE];
  int64_t a_off[AE];
  const int a_elems = 1 << g.a_tbits;
#pragma unroll
  for (int j = 0; j < AE; ++j) {
    const int e = tid + j * NT;
    a_sm[j] = -1;
    a_off[j] = 0;
    if (e < a_elems) {
      int r = 0, c = 0;
      int64_t off = 0;
      for (int t = 0; t < g.a_tbits; ++t)
        if ((e >> t) & 1) {
          const int s = g.a_tsel[t];
          if (s & 64) c |= 1 << (s & 63); else r |= 1 << (s & 63);
          off += (int64_t)1 << g.a_tpos[t];
        }
      a_sm[j] = c * TM + r;
      a_off[j] = off;
    }
  }
  int b_sm[BE];
  int64_t b_off[BE];
  const int b_elems = 1 << g.b_tbits;
#pragma unroll
  for (int j = 0; j < BE; ++j) {
    const int e = tid + j * NT;
    b_sm[j] = -1;
    b_off[j] = 0;
    if (e < b_elems) {
      int k = 0, n = 0;
      int64_t off = 0;
      for (int t = 0; t < g.b_tbits; ++t)
        if ((e >> t) & 1) {
          const int s = g.b_tsel[t];
          if (s & 64) k |= 1 << (s & 63); else n |= 1 << (s & 63);
          off += (int64_t)1 << g.b_tpos[t];
        }
      b_sm[j] = k * TN + n;
      b_off[j] = off;
    }
  }
  __syncthreads();

  const int nkc = 1 << (g.nk - g.tk);
  float am = 0.f;   // largest component written (for the FP16 split's scaling)
  for (int inst = bz; inst < g.n_inst; inst += gz) {
    const float2* A = g.A + inst_offset(inst, g.a_istride, g.a_bpos, g.nb) +
                      deposit_hi((uint64_t)bx, g.a_mpos, g.tm, g.nm);
    const float2* B = g.B + inst_offset(inst, g.b_istride, g.b_bpos, g.nb) +
                      deposit_hi((uint64_t)by, g.b_npos, g.tn, g.nn);
    float2* C = g.C + inst_offset(inst, g.c_istride, g.c_bpos, g.nb) +
                deposit_hi((uint64_t)bx, g.c_mpos, g.tm, g.nm) + deposit_hi((uint64_t)by, g.c_npos, g.tn, g.nn);
    float2 acc[RM][RN];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < RN; ++j) acc[i][j] = make_float2(0.f, 0.f);
    float2 ra[AE], rb[BE];
    auto load = [&](int kc) {
      const int64_t ka = deposit_hi((uint64_t)kc, g.a_kpos, g.tk, g.nk);
      const int64_t kb = deposit_hi((uint64_t)kc, g.b_kpos, g.tk, g.nk);
#pragma unroll
      for (int j = 0; j < AE; ++j)
        if (a_sm[j] >= 0) ra[j] = __ldg(A + ka + a_off[j]);
#pragma unroll
      for (int j = 0; j < BE; ++j)
        if (b_sm[j] >= 0) rb[j] = __ldg(B + kb + b_off[j]);
    };
    load(0);
    for (int kc = 0; kc < nkc; ++kc) {
      __syncthreads();
#pragma unroll
      for (int j = 0; j < AE; ++j)
        if (a_sm[j] >= 0) (&As[0][0])[a_sm[j]] = ra[j];
#pragma unroll
      for (int j = 0; j < BE; ++j)
        if (b_sm[j] >= 0) (&Bs[0][0])[b_sm[j]] = rb[j];
      __syncthreads();
      if (kc + 1 < nkc) load(kc + 1);
#pragma unroll 4
      for (int kk = 0; kk < TKv; ++kk) {
        float2 a[RM], b[RN];
#pragma unroll
        for (int i = 0; i < RM; ++i) a[i] = As[kk][tx + i * NTX];
#pragma unroll
        for (int j = 0; j < RN; ++j) b[j] = Bs[kk][ty + j * NTY];
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
          for (int j = 0; j < RN; ++j) {
            acc[i][j].x = fmaf(a[i].x, b[j].x, acc[i][j].x);
            acc[i][j].x = fmaf(-a[i].y, b[j].y, acc[i][j].x);
            acc[i][j].y = fmaf(a[i].x, b[j].y, acc[i][j].y);
            acc[i][j].y = fmaf(a[i].y, b[j].x, acc[i][j].y);
          }
      }
    }
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < RN; ++j) {
        const int r = tx + i * NTX, c = ty + j * NTY;
        if (r < TMv && c < TNv) {
          C[offCm[r] + offCn[c]] = acc[i][j];
          am = fmaxf(am, cabs_max(acc[i][j]));
        }
      }
  }
  if (g.amax_c) amax_update(g.amax_c, am);   // every thread reaches here (NT is a multiple of 32)
}

// One GEMM: grid (m tiles, n tiles, min(instances, 65535)).
template <int TM, int TN, int TK, int RM, int RN>
__global__ void __launch_bounds__((TM / RM) * (TN / RN))
k_cgemm_simt(const GemmArgs g) {
  __shared__ SimtSmem<TM, TN, TK> sm;
  simt_tile<TM, TN, TK, RM, RN>(g, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.z, sm);
}

// Several independent GEMMs in one launch (a group of small steps that
// neither read nor write what another of the group writes): block b runs
// block b - start[i] of GEMM i, where start[i] <= b < start[i + 1] (start[n]
// is the grid size), decoded as (m tile, n tile, instance) with the m tile
// fastest, exactly as that GEMM's own grid would, with that GEMM's tiling
// tiling[i] (0: 64x64, 1: 128x16, 2: 256x4; all three use 256 threads).
__global__ void __launch_bounds__(256)
k_cgemm_simt_multi(const GemmArgs* __restrict__ gs, const int32_t* __restrict__ start,
                   const int8_t* __restrict__ tiling, int32_t n) {
  __shared__ GemmArgs sg;
  __shared__ int s_i;
  __shared__ union {   // one tiling per block: their tiles share the space
    SimtSmem<64, 64, 8> t0;
    SimtSmem<128, 16, 16> t1;
    SimtSmem<256, 4, 16> t2;
  } sm;
  const int b = blockIdx.x;
  if (threadIdx.x == 0) {
    int i = 0;
    while (i + 1 < n && start[i + 1] <= b) ++i;
    s_i = i;
  }
  __syncthreads();
  const int i = s_i;
  {
    const int words = (int)(sizeof(GemmArgs) / 4);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(gs + i);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sg);
    for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
  }
  __syncthreads();
  const int gx = 1 << (sg.nm - sg.tm), gy = 1 << (sg.nn - sg.tn);
  const int gz = sg.n_inst < 65535 ? sg.n_inst : 65535;
  const int lb = b - start[i];
  const int bx = lb % gx, by = (lb / gx) % gy, bz = lb / (gx * gy);
  switch (tiling[i]) {   // block-uniform
    case 0:
      simt_tile<64, 64, 8, 4, 4>(sg, bx, by, bz, gz, sm.t0);
      break;
    case 1:
      simt_tile<128, 16, 16, 4, 2>(sg, bx, by, bz, gz, sm.t1);
      break;
    default:
      simt_tile<256, 4, 16, 4, 1>(sg, bx, by, bz, gz, sm.t2);
      break;
  }
}

}  // namespace tnx
