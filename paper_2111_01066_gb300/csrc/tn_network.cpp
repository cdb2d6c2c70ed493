// Circuit -> tensor network (SI, TN section and figure S2), host tensor
// arithmetic used by the simplification pass, and the error channel of the ABI.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <unordered_map>

#include "tn_internal.h"

namespace tnx {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }
void fail(tn_status code, const std::string& msg) { throw TnError{code, msg}; }

// Deposit the bits of `x` at the given positions: sum_i bit_i(x) 2^{pos[i]}.
static inline uint64_t deposit(uint64_t x, const std::vector<int>& pos) {
  uint64_t r = 0;
  for (size_t i = 0; i < pos.size(); ++i)
    if ((x >> i) & 1) r |= uint64_t(1) << pos[i];
  return r;
}

HTensor hcontract(const HTensor& a, const HTensor& b, const std::vector<char>* keep) {
  // shared wires are summed, except those marked in `keep`, which stay as one
  // index of the result with both operands taken at the same value (diagonal)
  std::vector<int> sh_a, sh_b, fa_pos, fb_pos, kb_of_fa;
  for (int i = 0; i < a.rank(); ++i) {
    auto it = std::find(b.wires.begin(), b.wires.end(), a.wires[i]);
    const bool kept = keep && (*keep)[a.wires[i]];
    if (it != b.wires.end() && !kept) {
      sh_a.push_back(i);
      sh_b.push_back(int(it - b.wires.begin()));
    } else {
      fa_pos.push_back(i);
      kb_of_fa.push_back(it != b.wires.end() ? int(it - b.wires.begin()) : -1);
    }
  }
  for (int j = 0; j < b.rank(); ++j)
    if (std::find(a.wires.begin(), a.wires.end(), b.wires[j]) == a.wires.end()) fb_pos.push_back(j);
  HTensor c;
  for (int i : fa_pos) c.wires.push_back(a.wires[i]);
  for (int j : fb_pos) c.wires.push_back(b.wires[j]);
  if (c.rank() > 30) fail(TN_ERR_UNSUPPORTED, "host pre-contraction result too large");
  const uint64_t nfa = uint64_t(1) << fa_pos.size(), nfb = uint64_t(1) << fb_pos.size();
  const uint64_t nsh = uint64_t(1) << sh_a.size();
  c.data.assign(nfa * nfb, cd(0, 0));
  std::vector<uint64_t> sa(nsh), sb(nsh);
  for (uint64_t s2 = 0; s2 < nsh; ++s2) {
    sa[s2] = deposit(s2, sh_a);
    sb[s2] = deposit(s2, sh_b);
  }
  for (uint64_t j = 0; j < nfb; ++j) {
    const uint64_t bj = deposit(j, fb_pos);
    for (uint64_t i = 0; i < nfa; ++i) {
      const uint64_t ai = deposit(i, fa_pos);
      uint64_t bk = 0;   // kept wires: B takes the value A's index carries
      for (size_t t = 0; t < fa_pos.size(); ++t)
        if (kb_of_fa[t] >= 0 && ((i >> t) & 1)) bk |= uint64_t(1) << kb_of_fa[t];
      cd acc(0, 0);
      for (uint64_t s2 = 0; s2 < nsh; ++s2) acc += a.data[ai | sa[s2]] * b.data[bj | bk | sb[s2]];
      c.data[i + nfa * j] = acc;
    }
  }
  return c;
}

HTensor hfix(const HTensor& t, int wire, int value) {
  auto it = std::find(t.wires.begin(), t.wires.end(), wire);
  if (it == t.wires.end()) return t;
  const int p = int(it - t.wires.begin());
  HTensor r;
  std::vector<int> keep;
  for (int i = 0; i < t.rank(); ++i)
    if (i != p) {
      keep.push_back(i);
      r.wires.push_back(t.wires[i]);
    }
  const uint64_t n = uint64_t(1) << keep.size();
  r.data.resize(n);
  const uint64_t fixed = uint64_t(value) << p;
  for (uint64_t i = 0; i < n; ++i) r.data[i] = t.data[deposit(i, keep) | fixed];
  return r;
}

HTensor hpermute(const HTensor& t, const std::vector<int>& order) {
  // order[i] = wire id placed at new position i
  std::vector<int> src_pos;
  for (int w : order) {
    auto it = std::find(t.wires.begin(), t.wires.end(), w);
    if (it == t.wires.end()) fail(TN_ERR_PLAN, "internal: permute with unknown wire");
    src_pos.push_back(int(it - t.wires.begin()));
  }
  HTensor r;
  r.wires = order;
  const uint64_t n = uint64_t(1) << order.size();
  r.data.resize(n);
  for (uint64_t i = 0; i < n; ++i) r.data[i] = t.data[deposit(i, src_pos)];
  return r;
}

}  // namespace tnx

using namespace tnx;

extern "C" const char* tn_last_error(void) { return g_last_error.c_str(); }

extern "C" tn_status tn_network_from_circuit(const tn_circuit* c, tn_network_t** out) {
  try {
    clear_error();
    if (!c || !out) fail(TN_ERR_ARG, "tn_network_from_circuit: NULL argument");
    *out = nullptr;
    if (c->n_qubits < 1 || c->n_qubits > 64) fail(TN_ERR_ARG, "n_qubits must be in [1, 64]");
    if (c->n_gates < 0) fail(TN_ERR_ARG, "n_gates must be >= 0");
    if (c->n_gates > 0 && (!c->gate_qubits || !c->gate_matrices))
      fail(TN_ERR_ARG, "gate_qubits / gate_matrices must not be NULL");
    auto* h = new (std::nothrow) tn_network_s;
    if (!h) fail(TN_ERR_OOM, "host allocation failed");
    Network& net = h->net;
    const int n = c->n_qubits;
    net.n_qubits = n;
    std::vector<int> cur(n);
    net.gates_per_qubit.assign(n, 0);
    auto new_wire = [&](int q, int t) {
      net.labels.push_back({q, t});
      return int(net.labels.size()) - 1;
    };
    for (int q = 0; q < n; ++q) {
      cur[q] = new_wire(q, 0);
      net.input_wire.push_back(cur[q]);
    }
    const double* m = c->gate_matrices;
    for (int g = 0; g < c->n_gates; ++g) {
      const int q0 = c->gate_qubits[2 * g], q1 = c->gate_qubits[2 * g + 1];
      if (q0 < 0 || q0 >= n || q1 < -1 || q1 >= n || q1 == q0) {
        delete h;
        fail(TN_ERR_ARG, "gate " + std::to_string(g) + ": qubit index out of range or repeated");
      }
      HTensor t;
      if (q1 < 0) {
        // legs (out, in); entries U[out][in] from row-major interleaved complex128
        const int in = cur[q0];
        const int o = new_wire(q0, ++net.gates_per_qubit[q0]);
        t.wires = {o, in};
        t.data.resize(4);
        for (int r = 0; r < 2; ++r)
          for (int col = 0; col < 2; ++col)
            t.data[r + 2 * col] = cd(m[2 * (2 * r + col)], m[2 * (2 * r + col) + 1]);
        cur[q0] = o;
        m += 8;
      } else {
        // legs (out0, out1, in0, in1); entries U[2 out0 + out1][2 in0 + in1]
        const int i0 = cur[q0], i1 = cur[q1];
        const int o0 = new_wire(q0, ++net.gates_per_qubit[q0]);
        const int o1 = new_wire(q1, ++net.gates_per_qubit[q1]);
        t.wires = {o0, o1, i0, i1};
        t.data.resize(16);
        for (int a0 = 0; a0 < 2; ++a0)
          for (int a1 = 0; a1 < 2; ++a1)
            for (int b0 = 0; b0 < 2; ++b0)
              for (int b1 = 0; b1 < 2; ++b1) {
                const int r = 2 * a0 + a1, col = 2 * b0 + b1;
                t.data[a0 + 2 * a1 + 4 * b0 + 8 * b1] =
                    cd(m[2 * (4 * r + col)], m[2 * (4 * r + col) + 1]);
              }
        cur[q0] = o0;
        cur[q1] = o1;
        m += 32;
      }
      for (const cd& v : t.data)
        if (!std::isfinite(v.real()) || !std::isfinite(v.imag())) {
          delete h;
          fail(TN_ERR_ARG, "gate " + std::to_string(g) + ": non-finite matrix entry");
        }
      net.gates.push_back(std::move(t));
    }
    net.output_wire = cur;
    *out = h;
    return TN_OK;
  } catch (const TnError& e) {
    set_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return TN_ERR_OOM;
  }
}

extern "C" tn_status tn_network_wire_counts(const tn_network_t* h, int32_t* gpq, int32_t cap) {
  clear_error();
  if (!h || !gpq) {
    set_error("tn_network_wire_counts: NULL argument");
    return TN_ERR_ARG;
  }
  if (cap < h->net.n_qubits) {
    set_error("tn_network_wire_counts: cap smaller than n_qubits");
    return TN_ERR_ARG;
  }
  for (int q = 0; q < h->net.n_qubits; ++q) gpq[q] = h->net.gates_per_qubit[q];
  return TN_OK;
}

extern "C" void tn_network_destroy(tn_network_t* h) { delete h; }
