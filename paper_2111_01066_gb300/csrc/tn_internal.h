// Internal structures shared by the host planner and the device executor.
#pragma once

#include <bitset>
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "tn.h"

namespace tnx {

using cd = std::complex<double>;

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
void clear_error();
struct TnError {
  tn_status code;
  std::string msg;
};
[[noreturn]] void fail(tn_status code, const std::string& msg);

// ------------------------------------------------------------------ host tensors
// A dense complex tensor whose every index has dimension 2; wires[0] is the
// fastest index (column-major, as in the paper's SI figure S7 caption).
struct HTensor {
  std::vector<int> wires;
  std::vector<cd> data;
  int rank() const { return (int)wires.size(); }
};

HTensor hcontract(const HTensor& a, const HTensor& b,
                  const std::vector<char>* keep = nullptr);  // sum over shared wires not in keep
HTensor hfix(const HTensor& t, int wire, int value);        // index one wire at a value
HTensor hpermute(const HTensor& t, const std::vector<int>& order);  // new wire order

struct WireLabel {
  int q, t;
};

// tn_network_s: the circuit as one tensor per gate (SI, figure S2)
struct Network {
  int n_qubits = 0;
  std::vector<WireLabel> labels;   // wire id -> (qubit, gate count so far)
  std::vector<HTensor> gates;
  std::vector<int> input_wire;     // per qubit: wire (q, 0)
  std::vector<int> output_wire;    // per qubit: wire (q, T_q)
  std::vector<int> gates_per_qubit;
};

// ------------------------------------------------------------------ plan
constexpr int MAXR = 48;   // bits per tensor index tracked by a step descriptor
constexpr int MAXFIX = 24; // fixed (sliced or closed-output) wires per leaf

// One pairwise contraction C[m, n] = sum_k A[m, k] B[k, n] over a batch of
// instances (SI, Eq. (2)).  Every index is a bit of an element offset: the
// m-th row of A starts at sum_i bit_i(m) 2^{a_mpos[i]} etc.  Positions at or
// above an operand's rank address its batch instances (slices of the chunk);
// batch bits carried by only one operand are folded into that operand's m or n
// bits, so only bits shared by A and B remain true batch bits (nb).
constexpr int MAXB = 16;
struct StepDesc {
  int64_t a_off, b_off, c_off;        // arena offsets in complex64 elements
  int64_t a_elems, b_elems, c_elems;  // elements of each operand over all its instances
  int32_t nm, nk, nn, nb;             // log2 of M, K, N and of the instance count
  int32_t nm_wires, nn_wires;         // m / n bits that are wires (the rest are batch bits)
  int32_t rank_a, rank_b, rank_c;     // per-slice ranks
  int32_t kernel;                     // kernel variant chosen by the executor
  int32_t a_node, b_node, c_node;     // node ids (leaves 0..L-1, step i's result L+i)
  int32_t dep_flags;                  // result depends on the slice id (bit 0), on closed output bits (bit 1)
  int32_t group;                      // steps with one group id >= 0 are consecutive, independent of each
                                      // other, and no output of one overlaps an operand of another: they
                                      // may run concurrently (small slice-dependent steps); -1 otherwise
  int8_t a_mpos[MAXR], a_kpos[MAXR], b_kpos[MAXR], b_npos[MAXR], c_mpos[MAXR], c_npos[MAXR];
  int8_t a_bpos[MAXB], b_bpos[MAXB], c_bpos[MAXB];
};

// One leaf tensor materialised per chunk by the leaf-select kernel.
struct LeafDesc {
  int64_t src_off;    // offset of the leaf's full data in the leaf buffer (elements)
  int64_t dst_off;    // arena offset of instance 0
  int32_t rank;       // planning wires kept (2^rank elements per instance)
  uint32_t bmask;     // batch (low slice) bits this leaf carries, as a mask over [0, b)
  int8_t bslice[MAXB];  // slice bit of the t-th batch bit in storage order (positions rank + t)
  int32_t nfixed;
  int8_t fixed_kind[MAXFIX];   // 0: slice bit, 1: closed-output qubit
  int8_t fixed_index[MAXFIX];  // slice bit j or qubit q
};

// Accumulation of the root tensor into the FP64 amplitudes.
struct RootDesc {
  int64_t off;
  int32_t rank;        // = number of open qubits
  uint32_t bmask;      // batch bits carried by the root (mask over [0, b))
  int8_t bslice[MAXB]; // slice bit of the t-th batch bit in storage order
  int8_t pos_of_open[64];  // root bit position of the j-th open qubit
};

struct PlanStats {
  double flops_slice = 0, bytes_slice = 0, flops_chunk = 0, bytes_chunk = 0;
  int log2_max = 0;
  int khist[40] = {0};
};

struct DeviceState;  // defined by the executor

struct Plan {
  tn_plan_opts opts{};
  int n_qubits = 0;
  std::vector<int> open_qubits;
  std::vector<WireLabel> sliced;       // slice bit j -> wire label
  int log2_batch = 0;                  // b: slices per chunk = 2^b
  int n_leaves = 0;
  std::vector<std::complex<float>> leaf_data;
  std::vector<LeafDesc> leaves;
  std::vector<float> leaf_amax;        // largest |re|, |im| of each leaf's data (FP16 scaling)
  std::vector<StepDesc> steps;
  std::vector<std::vector<int>> leaf_gates;   // per leaf: circuit gates absorbed into it
  RootDesc root{};
  int64_t arena_elems = 0;
  PlanStats stats;
  DeviceState* dev = nullptr;
  tn_status sticky = TN_OK;
  std::string sticky_msg;
};

Plan* build_plan(const Network& net, const tn_plan_opts& opts);
void destroy_device_state(Plan* p);

}  // namespace tnx

struct tn_network_s {
  tnx::Network net;
};
struct tn_plan_s {
  tnx::Plan plan;
};
