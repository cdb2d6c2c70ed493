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
  // FP16 split with power-of-two scaling (NULL when unused): max |re|, |im| of
  // A and B (written by their producers) and C's maximum, which this GEMM
  // records for its consumer
  const float* amax_a;
  const float* amax_b;
  float* amax_c;
};

static_assert(sizeof(GemmArgs) % 4 == 0, "GemmArgs is copied to shared memory in 4-byte words");

// Exponent s of the power-of-two scale 2^s that maps a tensor's largest
// component into [2^14, 2^15), inside the FP16 range (|s| <= 126; 0 when the
// maximum is zero, subnormal or not recorded).
__device__ __forceinline__ int fp16_scale_exp(const float* amax) {
  if (!amax) return 0;
  const int be = (int)((__float_as_uint(*amax) >> 23) & 255u);
  if (be == 0 || be == 255) return 0;
  const int s = 14 - (be - 127);
  return s < -126 ? -126 : (s > 126 ? 126 : s);
}
// 2^e for |e| <= 126, exact
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }
// Warp-collective: raise *amax_c to the warp's largest m (m >= 0; non-negative
// floats order like their bit patterns).
__device__ __forceinline__ void amax_update(float* amax_c, float m) {
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned*>(amax_c), __float_as_uint(m));
}
__device__ __forceinline__ float cabs_max(float2 v) { return fmaxf(fabsf(v.x), fabsf(v.y)); }

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
