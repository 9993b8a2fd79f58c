// Host planner: validation, greedy k-local fusion (Sec. "Circuit Splitting" circuit splitting, re-targeted to
// tiles of 2^k amplitudes), register phases and conflict-free shared-memory layouts.
#include "planner.hpp"

#include <algorithm>
#include <cstdio>
#include <set>
#include <sstream>

namespace qsim {

static bool is_1q(int t) { return t == QSIM_RX || t == QSIM_RY || t == QSIM_RZ || t == QSIM_H || t == QSIM_X; }
static bool is_rot(int t) { return t == QSIM_RX || t == QSIM_RY || t == QSIM_RZ; }
// gates the pass kernels apply unnormalised (their scale is applied later, see kRescaleEvery)
static bool is_scaled(int t) { return is_rot(t) || t == QSIM_H; }

int validate_gates(const qsim_gate* g, int n_gates, int n, std::vector<Gate>& out, int& n_params,
                   int& n_inputs, std::string& err) {
  char buf[256];
  out.clear();
  n_params = 0;
  n_inputs = 0;
  if (n < 1 || n > kMaxQubits) {
    snprintf(buf, sizeof buf, "n_qubits=%d outside [1, %d]", n, kMaxQubits);
    err = buf;
    return QSIM_ERR_UNSUPPORTED;
  }
  if (n_gates < 0 || (n_gates > 0 && g == nullptr)) {
    err = "gate list is NULL or n_gates < 0";
    return QSIM_ERR_ARG;
  }
  for (int i = 0; i < n_gates; i++) {
    const qsim_gate& x = g[i];
    Gate y{x.type, x.targets[0], x.targets[1], x.controls[0], x.controls[1], x.param};
    auto bad_q = [&](int q) { return q < 0 || q >= n; };
    if (x.type < QSIM_RX || x.type > QSIM_CZ) {
      snprintf(buf, sizeof buf, "gate %d: unknown type %d", i, x.type);
      err = buf;
      return QSIM_ERR_GATE;
    }
    if (is_1q(x.type)) {
      if (bad_q(x.targets[0]) || x.targets[1] != -1 || x.controls[0] != -1 || x.controls[1] != -1) {
        snprintf(buf, sizeof buf, "gate %d: single-qubit gate needs targets[0] in [0,%d) and all other slots -1", i, n);
        err = buf;
        return QSIM_ERR_QUBIT;
      }
    } else {
      if (bad_q(x.targets[0]) || bad_q(x.controls[0]) || x.targets[1] != -1 || x.controls[1] != -1 ||
          x.targets[0] == x.controls[0]) {
        snprintf(buf, sizeof buf, "gate %d: two-qubit gate needs distinct controls[0], targets[0] in [0,%d)", i, n);
        err = buf;
        return QSIM_ERR_QUBIT;
      }
    }
    if (is_rot(x.type)) {
      if (x.param == -1) {
        snprintf(buf, sizeof buf, "gate %d: rotation without a parameter", i);
        err = buf;
        return QSIM_ERR_PARAM;
      }
      // the kernels index params[param] and inputs[b][-2 - param]: refuse indices no real buffer has
      if (x.param >= kMaxParams || (x.param <= -2 && (int64_t)-2 - x.param >= kMaxInputs)) {
        snprintf(buf, sizeof buf, "gate %d: param=%d outside [-2 - %d, %d)", i, x.param, kMaxInputs - 1, kMaxParams);
        err = buf;
        return QSIM_ERR_PARAM;
      }
      if (x.param >= 0) n_params = std::max(n_params, x.param + 1);
      else n_inputs = std::max(n_inputs, -2 - x.param + 1);
    } else if (x.param != -1) {
      snprintf(buf, sizeof buf, "gate %d: non-parametric gate with param=%d (must be -1)", i, x.param);
      err = buf;
      return QSIM_ERR_PARAM;
    }
    out.push_back(y);
  }
  return QSIM_OK;
}

static void gate_qubits(const Gate& g, int q[2], int& nq) {
  nq = 0;
  q[nq++] = g.t0;
  if (g.c0 >= 0) q[nq++] = g.c0;
}

// Simple deterministic generator for the layout search.
struct Lcg {
  uint64_t s;
  uint32_t next() {
    s = s * 6364136223846793005ULL + 1442695040888963407ULL;
    return (uint32_t)(s >> 33);
  }
};

static int rank3(const uint32_t* v, int m) {
  // rank over GF(2) of m vectors of 3 bits
  uint32_t basis[3] = {0, 0, 0};
  int r = 0;
  for (int i = 0; i < m; i++) {
    uint32_t x = v[i];
    for (int b = 2; b >= 0; b--) {
      if (!((x >> b) & 1)) continue;
      if (!basis[b]) { basis[b] = x; r++; x = 0; break; }
      x ^= basis[b];
    }
  }
  return r;
}

// Lane tile bits of a phase: the (up to) 3 lowest thread bits (lanes 0..7 of a 16-byte wavefront).
static int lane_bits(const DevPhase& ph, int out[3]) {
  int m = std::min<int>(3, ph.n_tbits);
  for (int i = 0; i < m; i++) out[i] = ph.tbit[i];
  return m;
}

static bool layout_ok(const DevLayout& L, const int* lanes, int m, int w0) {
  uint32_t v[3];
  for (int i = 0; i < m; i++) {
    int j = lanes[i];
    uint32_t word = (1u << j) ^ L.m[j];
    v[i] = (word >> w0) & 7u;
  }
  return rank3(v, m) == m;
}

static void choose_layout(DevLayout& L, const DevPhase* a, const DevPhase* b, int k, int w0, Lcg&) {
  for (int j = 0; j < kMaxTileBits; j++) L.m[j] = 0;
  int la[3], lb[3], ma = 0, mb = 0;
  if (a) ma = lane_bits(*a, la);
  if (b) mb = lane_bits(*b, lb);
  // deterministic in the constraint (identical pass structures get identical layouts)
  uint64_t seed = 0x9E3779B97F4A7C15ULL ^ (uint64_t)(w0 * 131 + k);
  for (int i = 0; i < ma; i++) seed = seed * 1000003ULL + (uint64_t)(la[i] + 1);
  seed = seed * 1000003ULL + 77;
  for (int i = 0; i < mb; i++) seed = seed * 1000003ULL + (uint64_t)(lb[i] + 1);
  Lcg rng{seed};
  auto ok = [&]() { return (!a || layout_ok(L, la, ma, w0)) && (!b || layout_ok(L, lb, mb, w0)); };
  if (ok()) return;
  const int src_min = w0 + 3;   // bits at or above the window may drive the XOR
  std::vector<int> srcs;
  for (int i = 0; i < ma; i++) if (la[i] >= src_min) srcs.push_back(la[i]);
  for (int i = 0; i < mb; i++) if (lb[i] >= src_min) srcs.push_back(lb[i]);
  std::sort(srcs.begin(), srcs.end());
  srcs.erase(std::unique(srcs.begin(), srcs.end()), srcs.end());
  for (int trial = 0; trial < 4096; trial++) {
    for (int j : srcs) L.m[j] = (uint8_t)((rng.next() & 7u) << w0);
    if (ok()) return;
  }
  for (int j = 0; j < kMaxTileBits; j++) L.m[j] = 0;   // fall back to the identity (correct, slower)
  (void)k;
}

int64_t tile_element_index(const DevPass& p, int64_t tile, int64_t e) {
  int64_t x = 0;
  for (int j = 0; j < p.k; j++)
    if ((e >> j) & 1) x |= (int64_t)1 << p.L[j];
  for (int j = 0; j < p.n_nonlocal; j++)
    if ((tile >> j) & 1) x |= (int64_t)1 << p.nonlocal[j];
  return x;
}

static int build_phases(Schedule& s, PassPlan& pp, DevPass& d, bool grads, int w0, Lcg& rng, std::string& err) {
  const int n = s.n, k = d.k, R = d.R;
  int tb_of_q[kMaxQubits];
  for (int q = 0; q < n; q++) tb_of_q[q] = -1;
  for (int j = 0; j < k; j++) tb_of_q[d.Q[j]] = j;
  d.phase0 = (int)s.phases.size();
  d.op0 = (int)s.ops.size();
  d.lay0 = (int)s.layouts.size();
  std::vector<int> remaining = pp.gates;
  int gslot = 0;
  int since_scale = 0;   // unnormalised ops since the pass start or the last K_SCALE
  // The first and the last register phase move their amplitudes straight between registers and global
  // memory: the first in the pass's input layout, the last in its output layout. The tile bits at
  // physical bits 1..3 of that layout (the low bits of a contiguous run) lead the phase's thread bits,
  // so lanes 0..7 of a warp cover one contiguous 128-byte run.
  std::vector<int> fin, fout;
  if (k - R >= 3)
    for (int b = 1; b <= 3 && b < s.c; b++)
      for (int j = 0; j < k; j++) {
        if (d.L[j] == b) fin.push_back(j);
        if (d.Lo[j] == b) fout.push_back(j);
      }
  auto in_list = [](const std::vector<int>& v, int x) { return std::find(v.begin(), v.end(), x) != v.end(); };
  auto excluded = [&](int tb, bool edge) { return edge && in_list(fin, tb); };
  // front: tile bits that must be the phase's leading thread bits (and so not register bits)
  auto make_phase = [&](std::vector<int> regs, const std::vector<int>& taken, const std::vector<int>* front) {
    for (int j = k - 1; j >= 0 && (int)regs.size() < R; j--)
      if (!in_list(regs, j) && !(front && in_list(*front, j))) regs.push_back(j);
    for (int j = k - 1; j >= 0 && (int)regs.size() < R; j--)   // small tiles: any bit
      if (!in_list(regs, j)) regs.push_back(j);
    std::sort(regs.begin() + 1, regs.end());
    DevPhase ph{};
    for (int i = 0; i < R; i++) ph.rbit[i] = (uint8_t)regs[i];
    int nt = 0;
    if (front)
      for (int j : *front)
        if (!in_list(regs, j)) ph.tbit[nt++] = (uint8_t)j;
    for (int j = 0; j < k; j++)
      if (!in_list(regs, j) && !(front && in_list(*front, j))) ph.tbit[nt++] = (uint8_t)j;
    ph.n_tbits = (uint8_t)nt;
    ph.op_begin = (int)s.ops.size();
    auto reg_of = [&](int tb) {
      for (int i = 0; i < R; i++)
        if (regs[i] == tb) return i;
      return -1;
    };
    for (int gi : taken) {
      const Gate& g = s.gates[gi];
      if (is_scaled(g.type) && since_scale == kRescaleEvery) {
        DevOp sc{};
        sc.kind = K_SCALE;
        sc.gate = -1;
        sc.gslot = -1;
        s.ops.push_back(sc);
        since_scale = 0;
      }
      since_scale += is_scaled(g.type);
      DevOp op{};
      op.gate = gi;
      op.gslot = -1;
      int ta = tb_of_q[g.t0];
      int ra = reg_of(ta);
      switch (g.type) {
        case QSIM_RY: op.kind = K_RY_R; op.a = (uint8_t)ra; break;
        case QSIM_RX: op.kind = K_RX_R; op.a = (uint8_t)ra; break;
        case QSIM_H: op.kind = K_H_R; op.a = (uint8_t)ra; break;
        case QSIM_X: op.kind = K_X_R; op.a = (uint8_t)ra; break;
        case QSIM_RZ:
          if (ra >= 0) { op.kind = K_RZ_R; op.a = (uint8_t)ra; }
          else { op.kind = K_RZ_T; op.a = (uint8_t)ta; }
          break;
        case QSIM_CNOT: {
          int tc = tb_of_q[g.c0], rc = reg_of(tc);
          op.a = (uint8_t)ra;
          if (rc >= 0) { op.kind = K_CNOT_RR; op.b = (uint8_t)rc; }
          else { op.kind = K_CNOT_RT; op.b = (uint8_t)tc; }
          break;
        }
        case QSIM_CZ: {
          int tc = tb_of_q[g.c0], rc = reg_of(tc);
          if (ra >= 0 && rc >= 0) { op.kind = K_CZ_RR; op.a = (uint8_t)ra; op.b = (uint8_t)rc; }
          else if (ra >= 0) { op.kind = K_CZ_RT; op.a = (uint8_t)ra; op.b = (uint8_t)tc; }
          else if (rc >= 0) { op.kind = K_CZ_RT; op.a = (uint8_t)rc; op.b = (uint8_t)ta; }
          else { op.kind = K_CZ_TT; op.a = (uint8_t)ta; op.b = (uint8_t)tc; }
          break;
        }
      }
      if (is_rot(g.type)) {
        op.rot = 1;
        op.gslot = gslot++;
        if (grads) {
          s.grad_gate.push_back(gi);
          s.grad_pass.push_back((int)(&pp - &s.passes[0]));
          s.grad_slot.push_back(op.gslot);
        }
      }
      s.ops.push_back(op);
    }
    ph.op_end = (int)s.ops.size();
    s.phases.push_back(ph);
  };
  bool first = true;
  while (!remaining.empty() || first) {
    std::vector<int> regs = {0};   // tile bit 0 is always a register bit
    std::set<int> blocked;
    std::vector<int> taken, rest;
    for (int gi : remaining) {
      const Gate& g = s.gates[gi];
      int q[2], nq;
      gate_qubits(g, q, nq);
      bool blk = false;
      for (int i = 0; i < nq; i++) blk |= blocked.count(q[i]) > 0;
      if (blk) {
        for (int i = 0; i < nq; i++) blocked.insert(q[i]);
        rest.push_back(gi);
        continue;
      }
      std::vector<int> need;
      if (g.type == QSIM_RX || g.type == QSIM_RY || g.type == QSIM_H || g.type == QSIM_X || g.type == QSIM_CNOT)
        need.push_back(tb_of_q[g.t0]);
      bool ok = true;
      for (int t : need) ok = ok && !excluded(t, first);
      std::vector<int> merged = regs;
      for (int t : need)
        if (std::find(merged.begin(), merged.end(), t) == merged.end()) merged.push_back(t);
      if (ok && (int)merged.size() <= R) {
        regs = merged;
        taken.push_back(gi);
      } else {
        for (int i = 0; i < nq; i++) blocked.insert(q[i]);
        rest.push_back(gi);
      }
    }
    const bool last = rest.empty();
    // the first phase loads in the input layout; a last phase also stores in the output layout when
    // its registers allow (else an op-free closing phase does, below)
    const std::vector<int>* front = first ? &fin : nullptr;
    if (last && !first) {
      bool viol = false;
      for (int t : regs) viol = viol || in_list(fout, t);
      if (!viol) front = &fout;
    }
    make_phase(regs, taken, front);
    first = false;
    remaining = rest;
  }
  // the last phase stores to global memory: add an op-free phase unless its leading thread bits are
  // the output layout's run
  if (!fout.empty()) {
    const DevPhase& lp = s.phases.back();
    bool ok = lp.n_tbits >= (int)fout.size();
    for (size_t i = 0; ok && i < fout.size(); i++) ok = lp.tbit[i] == fout[i];
    if (!ok) make_phase({0}, {}, &fout);
  }
  d.n_phases = (int)s.phases.size() - d.phase0;
  d.n_ops = (int)s.ops.size() - d.op0;
  d.n_gslots = gslot;
  // layouts: layout i sits between phase i-1 and phase i
  for (int i = 0; i <= d.n_phases; i++) {
    const DevPhase* a = i > 0 ? &s.phases[d.phase0 + i - 1] : nullptr;
    const DevPhase* b = i < d.n_phases ? &s.phases[d.phase0 + i] : nullptr;
    DevLayout L{};
    choose_layout(L, a, b, k, w0, rng);
    s.layouts.push_back(L);
  }
  return QSIM_OK;
}

int build_schedule(const std::vector<Gate>& gates, int n, const qsim_plan_opts& o, int R_fwd, int R_bwd,
                   Schedule& s, std::string& err, bool rotate_low) {
  s = Schedule{};
  s.n = n;
  s.gates = gates;
  s.dtype = o.dtype;
  s.mode = o.mode;
  s.max_regs = o.max_regs;
  s.pauli_frame = o.pauli_frame == 1 && o.mode == QSIM_FUSED;
  s.packed_bwd = s.pauli_frame && o.dtype == QSIM_C64 && o.scalar_bwd == 0;
  s.merge_diag = s.pauli_frame && o.split_diagonal == 0;
  int k = o.k > 0 ? o.k : 12;
  int c = o.contiguous_bits > 0 ? o.contiguous_bits : 4;
  if (k > kMaxTileBits) {
    err = "k larger than the supported tile (16 qubits)";
    return QSIM_ERR_UNSUPPORTED;
  }
  k = std::min(k, n);
  c = std::min(c, k);
  if (n >= 2 && k < std::min(n, c + 2)) {
    err = "k too small: need k >= contiguous_bits + 2";
    return QSIM_ERR_ARG;
  }
  int R = std::min(R_fwd, k);
  int Rb = std::min(R_bwd, k);
  s.k = k;
  s.R = R;
  s.Rb = Rb;
  s.c = c;
  int G = (int)gates.size();
  for (auto& g : gates) {
    if (is_rot(g.type)) {
      if (g.param >= 0) s.n_params = std::max(s.n_params, g.param + 1);
      else s.n_inputs = std::max(s.n_inputs, -2 - g.param + 1);
    }
  }
  if (o.mode == QSIM_PER_GATE) {
    // one pass per gate; only the gate list and gradient slots are used by the per-gate kernels
    for (int i = 0; i < G; i++) {
      PassPlan pp;
      pp.gates.push_back(i);
      pp.dev.k = 0;
      pp.dev.n_gslots = is_rot(gates[i].type) ? 1 : 0;
      pp.dev.gpart_offset = s.total_gslots;
      pp.devb = pp.dev;
      if (is_rot(gates[i].type)) {
        s.grad_gate.push_back(i);
        s.grad_pass.push_back(i);
        s.grad_slot.push_back(0);
      }
      s.total_gslots += pp.dev.n_gslots;
      s.passes.push_back(pp);
    }
    return QSIM_OK;
  }
  // ---- greedy k-local fusion, per-wire order preserved, with a rotating coalescing set.
  // The c lowest physical index bits must be tile bits of every pass (runs of 2^c amplitudes give
  // coalesced accesses). Physical bit 0 always holds qubit n-1 (the pair in one 16-byte word). Bits
  // 1..c-1 are handed between passes to qubits local in both passes, picked by their next use, so
  // they stop occupying tile slots for qubits the circuit does not touch next: pass p writes its
  // output in the new layout, a qubit remap that costs no memory traffic of its own (the paper's
  // reshape that moves the group's qubits into their own dimension, Sec. "Circuit Splitting", done by
  // the store addressing). The last pass writes the canonical layout.
  std::vector<char> done(G, 0);
  int n_done = 0;
  if (o.product_prefix == 1) {
    // a single-qubit gate on a qubit that no two-qubit gate has touched yet acts on that qubit's |0>
    // factor alone: it joins the qubit's prefix and leaves the fused passes
    s.prefix.assign(n, {});
    std::vector<char> entangled(n, 0);
    for (int i = 0; i < G; i++) {
      const Gate& g = gates[i];
      if (is_1q(g.type)) {
        if (!entangled[g.t0]) {
          s.prefix[g.t0].push_back(i);
          done[i] = 1;
          n_done++;
        }
      } else {
        entangled[g.t0] = entangled[g.c0] = 1;
      }
    }
    s.has_prefix = n_done > 0;
    if (!s.has_prefix) s.prefix.clear();
  }
  std::vector<int> phys(n), at(n);   // current layout: logical qubit -> physical bit, and inverse
  for (int q = 0; q < n; q++) {
    phys[q] = n - 1 - q;
    at[n - 1 - q] = q;
  }
  const bool rotate = rotate_low && k >= 2 * c + 2;   // room for the carried low qubits plus the canonical ones
  std::set<int> canon_low;
  for (int b = 0; b < c; b++) canon_low.insert(n - 1 - b);
  auto greedy = [&](std::set<int> S, std::vector<char>& dn, std::vector<int>& took) {
    std::set<int> blocked;
    int n_scaled = 0;
    for (int i = 0; i < G; i++) {
      if (dn[i]) continue;
      int q[2], nq;
      gate_qubits(gates[i], q, nq);
      bool blk = false;
      for (int j = 0; j < nq; j++) blk |= blocked.count(q[j]) > 0;
      if (blk) {
        for (int j = 0; j < nq; j++) blocked.insert(q[j]);
        continue;
      }
      std::set<int> T = S;
      for (int j = 0; j < nq; j++) T.insert(q[j]);
      const bool sc = is_scaled(gates[i].type);
      if ((int)T.size() <= k && (!sc || n_scaled < kMaxScaledOpsPerPass)) {
        S = T;
        took.push_back(i);
        dn[i] = 1;
        n_scaled += sc;
      } else {
        for (int j = 0; j < nq; j++) blocked.insert(q[j]);
      }
    }
    return S;
  };
  auto set_out_layout = [&](DevPass& d) {   // output layout of a pass = the current layout
    for (int j = 0; j < d.k; j++) d.Lo[j] = (uint8_t)phys[d.Q[j]];
    for (int i = 0; i < d.n_nonlocal; i++) d.nonlocal_o[i] = (uint8_t)phys[d.QN[i]];
  };
  std::vector<int> prevS;
  s.passes.reserve(G + 1);
  while (n_done < G || s.passes.empty()) {
    if (rotate && !s.passes.empty()) {
      // hand physical bits 1..c-1 to the previous pass's qubits that are needed soonest
      std::vector<int> next_use(n, G);
      for (int i = G - 1; i >= 0; i--) {
        if (done[i]) continue;
        int q[2], nq;
        gate_qubits(gates[i], q, nq);
        for (int j = 0; j < nq; j++) next_use[q[j]] = i;
      }
      std::vector<int> cand;
      for (int q : prevS)
        if (q != at[0]) cand.push_back(q);
      std::stable_sort(cand.begin(), cand.end(), [&](int a, int b) {
        return next_use[a] != next_use[b] ? next_use[a] < next_use[b] : phys[a] < phys[b];
      });
      for (int b = 1; b < c; b++) {
        const int qn = cand[b - 1], qo = at[b], pb = phys[qn];
        phys[qn] = b;
        at[b] = qn;
        phys[qo] = pb;
        at[pb] = qo;
      }
    }
    if (!s.passes.empty()) set_out_layout(s.passes.back().dev);   // the previous pass writes this layout
    std::set<int> S0;
    for (int b = 0; b < c; b++) S0.insert(at[b]);
    std::vector<char> dn = done;
    std::vector<int> took;
    std::set<int> S = greedy(S0, dn, took);
    if (rotate && n_done + (int)took.size() == G) {
      // the last pass writes the canonical layout: its low qubits must be in the tile
      std::set<int> T = S;
      T.insert(canon_low.begin(), canon_low.end());
      if ((int)T.size() <= k) {
        S = T;
      } else {
        std::set<int> S1 = S0;
        S1.insert(canon_low.begin(), canon_low.end());
        dn = done;
        took.clear();
        S = greedy(S1, dn, took);
      }
    }
    if (took.empty() && n_done < G) {   // (a circuit whose gates all went to the prefix gets one empty pass)
      err = "internal: fusion made no progress";
      return QSIM_ERR_ARG;
    }
    done = dn;
    n_done += (int)took.size();
    PassPlan pp;
    pp.gates = took;
    // pad the local set to k qubits, lowest physical bits first
    for (int b = 0; b < n && (int)S.size() < k; b++) S.insert(at[b]);
    // tile bits: 0..c-1 = physical bits 0..c-1 of the input layout, then the rest by physical bit
    std::vector<int> Q;
    for (int b = 0; b < c; b++) Q.push_back(at[b]);
    std::vector<int> rest;
    for (int q : S)
      if (phys[q] >= c) rest.push_back(q);
    std::sort(rest.begin(), rest.end(), [&](int a, int b) { return phys[a] < phys[b]; });
    Q.insert(Q.end(), rest.begin(), rest.end());
    DevPass& d = pp.dev;
    d.k = k;
    d.R = R;
    for (int j = 0; j < k; j++) {
      d.Q[j] = (uint8_t)Q[j];
      d.L[j] = (uint8_t)phys[Q[j]];
      pp.local_qubits.push_back(Q[j]);
    }
    int nl = 0;
    for (int b = 0; b < n; b++)
      if (!S.count(at[b])) {
        d.QN[nl] = (uint8_t)at[b];
        d.nonlocal[nl++] = (uint8_t)b;
      }
    d.n_nonlocal = nl;
    d.tiles_per_sample = (int64_t)1 << nl;
    prevS = Q;
    s.passes.push_back(pp);
    if (G == 0) break;
  }
  // the last pass writes the canonical layout
  for (int q = 0; q < n; q++) {
    phys[q] = n - 1 - q;
    at[n - 1 - q] = q;
  }
  set_out_layout(s.passes.back().dev);
  const int w0 = (o.dtype == QSIM_C128) ? 0 : 1;
  Lcg rng{0x51ED270B5EEDULL};
  for (auto& pp : s.passes) {
    pp.devb = pp.dev;
    pp.devb.R = Rb;
    int rc = build_phases(s, pp, pp.dev, false, w0, rng, err);
    if (rc) return rc;
    // packed backward: one 16-byte word per amplitude (psi and lambda), like complex128
    rc = build_phases(s, pp, pp.devb, true, s.packed_bwd ? 0 : w0, rng, err);
    if (rc) return rc;
    pp.dev.gpart_offset = s.total_gslots;
    pp.devb.gpart_offset = s.total_gslots;
    s.total_gslots += pp.devb.n_gslots;
  }
  // prefix rotations are gradient occurrences too, computed from the prefix contraction (no pass, no slot)
  for (int q = 0; q < (int)s.prefix.size(); q++)
    for (int gi : s.prefix[q])
      if (is_rot(gates[gi].type)) {
        s.grad_gate.push_back(gi);
        s.grad_pass.push_back(-1);
        s.grad_slot.push_back(-1);
      }
  return QSIM_OK;
}

std::string describe_schedule(const Schedule& s) {
  static const char* kn[] = {"ry", "rx", "rz", "h", "x", "rz_t", "cx", "cx_t", "cz", "cz_t", "cz_tt", "scale"};
  std::ostringstream o;
  o << "{\"n\":" << s.n << ",\"k\":" << s.k << ",\"R\":" << s.R << ",\"Rb\":" << s.Rb << ",\"c\":" << s.c
    << ",\"mode\":" << s.mode << ",\"n_params\":" << s.n_params << ",\"n_inputs\":" << s.n_inputs
    << ",\"prefix\":[";
  for (size_t q = 0; q < s.prefix.size(); q++) {
    o << (q ? "," : "") << "[";
    for (size_t i = 0; i < s.prefix[q].size(); i++) o << (i ? "," : "") << s.prefix[q][i];
    o << "]";
  }
  o << "],\"passes\":[";
  for (size_t p = 0; p < s.passes.size(); p++) {
    const auto& pp = s.passes[p];
    const auto& d = pp.dev;
    if (p) o << ",";
    o << "{\"gates\":[";
    for (size_t i = 0; i < pp.gates.size(); i++) o << (i ? "," : "") << pp.gates[i];
    o << "],\"local_qubits\":[";
    for (size_t i = 0; i < pp.local_qubits.size(); i++) o << (i ? "," : "") << pp.local_qubits[i];
    o << "],\"L\":[";
    for (int j = 0; j < d.k; j++) o << (j ? "," : "") << (int)d.L[j];
    o << "],\"nonlocal\":[";
    for (int j = 0; j < d.n_nonlocal; j++) o << (j ? "," : "") << (int)d.nonlocal[j];
    o << "],\"Lo\":[";
    for (int j = 0; j < d.k; j++) o << (j ? "," : "") << (int)d.Lo[j];
    o << "],\"nonlocal_o\":[";
    for (int j = 0; j < d.n_nonlocal; j++) o << (j ? "," : "") << (int)d.nonlocal_o[j];
    o << "],\"QN\":[";
    for (int j = 0; j < d.n_nonlocal; j++) o << (j ? "," : "") << (int)d.QN[j];
    o << "],\"n_gslots\":" << d.n_gslots;
    for (int dir = 0; dir < 2; dir++) {
      const DevPass& D = dir == 0 ? pp.dev : pp.devb;
      o << (dir == 0 ? ",\"phases\":[" : ",\"bwd_phases\":[");
      for (int ph = 0; ph < D.n_phases; ph++) {
        const DevPhase& P = s.phases[D.phase0 + ph];
        if (ph) o << ",";
        o << "{\"rbits\":[";
        for (int i = 0; i < D.R; i++) o << (i ? "," : "") << (int)P.rbit[i];
        o << "],\"tbits\":[";
        for (int i = 0; i < P.n_tbits; i++) o << (i ? "," : "") << (int)P.tbit[i];
        o << "],\"ops\":[";
        for (int i = P.op_begin; i < P.op_end; i++) {
          const DevOp& op = s.ops[i];
          o << (i > P.op_begin ? "," : "") << "{\"kind\":\"" << kn[op.kind] << "\",\"gate\":" << op.gate
            << ",\"a\":" << (int)op.a << ",\"b\":" << (int)op.b << ",\"gslot\":" << op.gslot << "}";
        }
        o << "]}";
      }
      o << (dir == 0 ? "],\"layouts\":[" : "],\"bwd_layouts\":[");
      if (D.k > 0)
        for (int i = 0; i <= D.n_phases; i++) {
          const DevLayout& L = s.layouts[D.lay0 + i];
          o << (i ? "," : "") << "[";
          for (int j = 0; j < D.k; j++) o << (j ? "," : "") << (int)L.m[j];
          o << "]";
        }
      o << "]";
    }
    o << "}";
  }
  o << "]}";
  return o.str();
}

}  // namespace qsim
