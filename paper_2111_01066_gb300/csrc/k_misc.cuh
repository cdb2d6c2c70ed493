// Small kernels of the slice loop: leaf select (slicing, main text section II),
// FP64 slice sum into the amplitudes, chunk advance, XEB reduction (Eq. (1))
// and the standalone index permutation (SI Eq. (2)).
#pragma once
#include "kernels_common.cuh"
#include "tn_internal.h"

namespace tnx {

// Materialise every leaf of the chunk: the sliced wires take the bits of the
// slice id, the closed output wires the bits of the batch's bitstring.
__global__ void k_leaf_select(const float2* __restrict__ leaf_data, const LeafDesc* __restrict__ leaves,
                              int n_leaves, float2* __restrict__ arena, const ChunkParam* __restrict__ params,
                              const unsigned* __restrict__ counter) {
  const ChunkParam p = params[*counter];
  for (int li = blockIdx.x; li < n_leaves; li += gridDim.x) {
    const LeafDesc& d = leaves[li];
    const int rank = d.rank;
    const int64_t per = (int64_t)1 << rank;
    const int nbat = __popc(d.bmask);
    const int64_t total = per << nbat;
    for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
      const uint32_t inst = (uint32_t)(e >> rank);
      const int64_t i = e & (per - 1);
      uint64_t sid = p.slice_base;
      for (int t = 0; t < nbat; ++t) sid |= (uint64_t)((inst >> t) & 1u) << d.bslice[t];
      int64_t fix = 0;
      for (int f = 0; f < d.nfixed; ++f) {
        const int idx = d.fixed_index[f];
        const uint64_t v = d.fixed_kind[f] == 0 ? ((sid >> idx) & 1) : ((p.bitstring >> idx) & 1);
        fix |= (int64_t)v << f;
      }
      arena[d.dst_off + e] = leaf_data[d.src_off + fix * per + i];
    }
  }
}

// Slice sum of a chunk (main text, section II: the sliced network is the sum of
// the smaller networks), FP64, in two deterministic passes: k_root_partial sums
// the slices of group g (slices g*per .. g*per+per-1 of the chunk) for every
// amplitude j into part[g][j]; k_root_finish adds the groups in order into
// out[batch][j].  Slices outside the call's range are skipped.
__global__ void __launch_bounds__(256) k_root_partial(const float2* __restrict__ arena, const RootDesc r, int b,
                                                     int groups, double2* __restrict__ part,
                                                     const ChunkParam* __restrict__ params,
                                                     const unsigned* __restrict__ counter) {
  // the group's slices in rounds of 256: their instance offsets in the root
  // (or -1 outside the call's range) are found once per block, then every
  // thread adds its amplitudes over them with four independent FP64
  // accumulators (slice i of a round goes to accumulator i % 4), combined in a
  // fixed order, so the sum is deterministic.  256 threads, s_off has 256
  // entries: cnt <= 256 and its padding to a multiple of 4 stays <= 256
  __shared__ int64_t s_off[256];
  const ChunkParam p = params[*counter];
  const int k = r.rank;
  const int64_t nout = (int64_t)1 << k;
  const uint32_t per = (1u << b) / (uint32_t)groups;
  const int g = blockIdx.y;
  const int nbat = __popc(r.bmask);
  const int64_t j0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t jstep = (int64_t)gridDim.x * blockDim.x;
  // every thread of the block takes part in the rounds (the barriers) the same
  // number of times, even where it has no amplitude: the pass count depends
  // on the grid only
  const int my_n = j0 < nout ? (int)((nout - 1 - j0) / jstep) + 1 : 0;
  constexpr int MAXJ = 4;   // amplitudes per thread held in registers
  const int64_t max_n = (nout + jstep - 1) / jstep;
  const int passes = (int)((max_n + MAXJ - 1) / MAXJ);
  double ar[MAXJ][4], ai[MAXJ][4];
  int64_t ri[MAXJ];
  for (int pass = 0; pass < passes; ++pass) {
    const int jj0 = pass * MAXJ;
    const int nj = my_n - jj0 < 0 ? 0 : (my_n - jj0 < MAXJ ? my_n - jj0 : MAXJ);
#pragma unroll
    for (int t = 0; t < MAXJ; ++t) {
      ri[t] = 0;
      if (t < nj) {
        const int64_t j = j0 + (int64_t)(jj0 + t) * jstep;
        for (int q = 0; q < k; ++q)
          if ((j >> q) & 1) ri[t] |= (int64_t)1 << r.pos_of_open[q];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) ar[t][u] = ai[t][u] = 0.0;
    }
    for (uint32_t s0 = (uint32_t)g * per; s0 < (uint32_t)(g + 1) * per; s0 += 256) {
      const uint32_t cnt = min(256u, (uint32_t)(g + 1) * per - s0);
      const uint32_t cnt4 = (cnt + 3u) & ~3u;   // padded with -1 (no slice) to whole quadruples
      __syncthreads();
      if (threadIdx.x < cnt4) {
        const uint32_t sl = s0 + threadIdx.x;
        const uint64_t sid = p.slice_base + sl;
        int64_t o = -1;
        if (threadIdx.x < cnt && sid >= p.valid_lo && sid < p.valid_hi) {
          uint32_t inst = 0;
          for (int t = 0; t < nbat; ++t) inst |= ((sl >> r.bslice[t]) & 1u) << t;
          o = r.off + ((int64_t)inst << k);
        }
        s_off[threadIdx.x] = o;
      }
      __syncthreads();
      // four slices per pass, one per accumulator: four independent loads in flight
      for (uint32_t i = 0; i < cnt4; i += 4) {
        int64_t o[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) o[u] = s_off[i + u];
#pragma unroll
        for (int t = 0; t < MAXJ; ++t)
          if (t < nj) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (o[u] >= 0) {
                const float2 v = arena[o[u] + ri[t]];
                ar[t][u] += (double)v.x;
                ai[t][u] += (double)v.y;
              }
          }
      }
    }
#pragma unroll
    for (int t = 0; t < MAXJ; ++t)
      if (t < nj) {
        const int64_t j = j0 + (int64_t)(jj0 + t) * jstep;
        part[(int64_t)g * nout + j] = make_double2((ar[t][0] + ar[t][1]) + (ar[t][2] + ar[t][3]),
                                                   (ai[t][0] + ai[t][1]) + (ai[t][2] + ai[t][3]));
      }
  }
}

__global__ void k_root_finish(const double2* __restrict__ part, int groups, int k,
                              const ChunkParam* __restrict__ params, const unsigned* __restrict__ counter) {
  const ChunkParam p = params[*counter];
  double* __restrict__ out = p.out;
  const int64_t nout = (int64_t)1 << k;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nout;
       j += (int64_t)gridDim.x * blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (int g = 0; g < groups; ++g) {
      const double2 v = part[(int64_t)g * nout + j];
      sr += v.x;
      si += v.y;
    }
    double* o = out + 2 * (p.out_index * nout + j);
    o[0] += sr;
    o[1] += si;
  }
}

__global__ void k_advance(unsigned* counter) { *counter += 1u; }

// Largest |re|, |im| over n complex values, raised into *out (which the caller
// zeroes first): the FP16 split's scale of an operand without a producer.
__global__ void k_amax(const float2* __restrict__ x, int64_t n, float* out) {
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, cabs_max(x[i]));
  amax_update(out, m);   // blockDim is a multiple of 32
}

// Frugal rejection sampling (main text, section III): sample s walks its
// draws t, draw t proposing batch member cand[s][t] with uniform u[s][t]; the
// first draw with u * M < 2^n |a|^2 is the sample.  Every draw is tested in
// parallel and the smallest accepted t per sample kept.  The products are
// rounded separately (no fused multiply-add), as the decision's definition
// states them.  A candidate outside [0, count) is skipped and flagged.
__global__ void k_frugal(const double2* __restrict__ a, int64_t count, int n_qubits, double m_bound,
                         const int64_t* __restrict__ cand, const double* __restrict__ u, int64_t n_draws,
                         int64_t n_samples, unsigned long long* first, int32_t* bad) {
  const int64_t total = n_draws * n_samples;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = cand[i];
    if (c < 0 || c >= count) {
      atomicExch(bad, 1);
      continue;
    }
    const double2 v = a[c];
    const double p = __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y));
    if (__dmul_rn(u[i], m_bound) < ldexp(p, n_qubits))
      atomicMin(first + i / n_draws, (unsigned long long)(i % n_draws));
  }
}

// sum_i |a_i|^2 in FP64 (one block; count is small)
__global__ void k_xeb_sum(const double2* __restrict__ a, int64_t n, double* __restrict__ out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 v = a[i];
    s = fma(v.x, v.x, s);
    s = fma(v.y, v.y, s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

struct PermArgs {
  int8_t src_pos[KMAXR];  // output bit p <- input bit src_pos[p]
  // tiled variant: the tile's bits (input positions), in input order; for each
  // tile bit its output position; the non-tile bits (input order) and theirs
  int32_t nt;             // tile bits (<= 10)
  int8_t t_in[10], t_out[10];
  int32_t nr;             // remaining bits
  int8_t r_in[KMAXR], r_out[KMAXR];
  int32_t t_out_order[10];  // tile bits sorted by output position (indices into t_*)
};

// Standalone permutation: one thread per output element (coalesced writes,
// gathered reads); used for small ranks.
__global__ void k_permute_gather(const float2* __restrict__ in, float2* __restrict__ out, int rank,
                                 const PermArgs pa, int64_t total) {
  const int64_t mask = ((int64_t)1 << rank) - 1;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = idx & mask;
    int64_t src = 0;
    for (int p = 0; p < rank; ++p)
      if ((o >> p) & 1) src |= (int64_t)1 << pa.src_pos[p];
    out[idx] = __ldg(in + (idx - o) + src);
  }
}

// Tiled permutation (SI Eq. (2) as a standalone pass): a tile holds every
// combination of nt <= 10 tile bits: the input's lowest bits and the input bits
// that feed the output's lowest positions (so reads and writes both run along
// memory).  Threads read the tile in input order into shared memory and write
// it back in output order; the remaining nr bits select the tile.  Each
// thread's in-tile offsets are fixed, so they are computed once; a tile's base
// is a one-bit-per-lane warp sum.
__global__ void __launch_bounds__(256) k_permute_tiled(const float2* __restrict__ in, float2* __restrict__ out,
                                                       int rank, const PermArgs pa, int64_t n_tiles_per_inst,
                                                       int64_t n_inst) {
  __shared__ float2 tile[1024];
  const int tsz = 1 << pa.nt;
  const int lane = threadIdx.x & 31;
  int64_t ioff[4], ooff[4];
  int sidx[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int e = threadIdx.x + 256 * j;   // element e in input order, element e in output order
    ioff[j] = -1;
    ooff[j] = 0;
    sidx[j] = 0;
    if (e < tsz) {
      int64_t io = 0, oo = 0;
      int si = 0;
      for (int q = 0; q < pa.nt; ++q)
        if ((e >> q) & 1) {
          io += (int64_t)1 << pa.t_in[q];
          const int i = pa.t_out_order[q];
          si |= 1 << i;
          oo += (int64_t)1 << pa.t_out[i];
        }
      ioff[j] = io;
      ooff[j] = oo;
      sidx[j] = si;
    }
  }
  const int64_t total = n_tiles_per_inst * n_inst;
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
    const int64_t inst = t >> pa.nr;
    const int64_t r = t & (n_tiles_per_inst - 1);
    int64_t bi = 0, bo = 0;
    for (int q0 = 0; q0 < pa.nr; q0 += 32) {
      const int q = q0 + lane;
      int64_t vi = 0, vo = 0;
      if (q < pa.nr && ((r >> q) & 1)) {
        vi = (int64_t)1 << pa.r_in[q];
        vo = (int64_t)1 << pa.r_out[q];
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        vi += __shfl_xor_sync(0xffffffffu, vi, o);
        vo += __shfl_xor_sync(0xffffffffu, vo, o);
      }
      bi += vi;
      bo += vo;
    }
    const int64_t ib = (inst << rank) + bi, ob = (inst << rank) + bo;
    // tile slot of element e: e ^ (bits 5-9 of e), so that runs along either
    // order spread over the shared-memory banks
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int e = threadIdx.x + 256 * j;
      if (ioff[j] >= 0) tile[e ^ ((e >> 5) & 31)] = __ldg(in + ib + ioff[j]);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (ioff[j] >= 0) out[ob + ooff[j]] = tile[sidx[j] ^ ((sidx[j] >> 5) & 31)];
    __syncthreads();
  }
}

}  // namespace tnx
