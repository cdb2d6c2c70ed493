// Device-side descriptors and helpers shared by the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tnx {

// Per-chunk parameters, read by the kernels from device memory at
// params[*counter] so that one captured launch sequence serves every chunk.
struct ChunkParam {
  uint64_t slice_base;   // first slice id of the chunk (aligned to 2^b)
  uint64_t valid_lo;     // slices [valid_lo, valid_hi) of the chunk are summed
  uint64_t valid_hi;
  uint64_t bitstring;    // closed output bits of the batch
  int64_t out_index;     // batch index into the output amplitudes
  double* out;           // the call's output amplitudes (complex128)
};

// Launch arguments of one gathered complex GEMM (one plan step or one
// tn_contract_pair call).  C[m, n] = sum_k A[m, k] B[k, n] for every batch
// instance; operand element offsets are sums of 2^position over set bits.
constexpr int KMAXR = 48;
constexpr int KMAXB = 16;
constexpr int KTB = 24;   // tile bits per operand tile
struct GemmArgs {
  const float2* A;
  const float2* B;
  float2* C;
  // instance i of a batch starts at i * istride + sum_j bit_j(i) 2^{bpos[j]}
  int64_t a_istride, b_istride, c_istride;
  int32_t n_inst;                  // batch instances (grid z)
  int32_t nb;                      // bits of the instance index deposited through *_bpos
  int32_t nm, nk, nn;              // log2 M, K, N
  int32_t tm, tk, tn;              // log2 of the tile extents actually used
  // tile decode in memory-position order: *_tsel[t] = index | (64 if a k bit)
  int32_t a_tbits, b_tbits;
  int8_t a_tpos[KTB], a_tsel[KTB];
  int8_t b_tpos[KTB], b_tsel[KTB];
  // all bit positions (tile bits first)
  int8_t a_mpos[KMAXR], a_kpos[KMAXR], b_kpos[KMAXR], b_npos[KMAXR], c_mpos[KMAXR], c_npos[KMAXR];
  int8_t a_bpos[KMAXB], b_bpos[KMAXB], c_bpos[KMAXB];
};

__device__ __forceinline__ uint32_t pext_u32(uint32_t x, uint32_t mask) {
  uint32_t r = 0, k = 0;
  while (mask) {
    const uint32_t low = mask & (0u - mask);
    if (x & low) r |= 1u << k;
    ++k;
    mask ^= low;
  }
  return r;
}

// sum over bits i >= from of bit_{i-from}(x) << pos[i]
__device__ __forceinline__ int64_t deposit_hi(uint64_t x, const int8_t* pos, int from, int to) {
  int64_t r = 0;
  for (int i = from; i < to; ++i)
    if ((x >> (i - from)) & 1) r += (int64_t)1 << pos[i];
  return r;
}

__device__ __forceinline__ int64_t inst_offset(uint32_t inst, int64_t istride, const int8_t* bpos, int nb) {
  int64_t r = (int64_t)inst * istride;
  for (int j = 0; j < nb; ++j)
    if ((inst >> j) & 1) r += (int64_t)1 << bpos[j];
  return r;
}

}  // namespace tnx
