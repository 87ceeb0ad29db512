// Circuit compiler: the dependency DAG, Algorithm 1 of the paper (Sec. 3) run with the
// tile bits as the local qubits, and the tile-pass scheduler that generalises it to
// multi-qubit reorderings folded into the pass addressing.
//
// Locality (Sec. 2, Appendix C): a gate needs "communication" -- here: cannot run inside a
// tile pass -- iff one of the qubits on which it acts non-diagonally sits outside the tile.
// Controls and diagonal factors on any qubit are constants of a tile block.
//
// Gate fusion (Sec. 1 cites fusing consecutive gates on a common qubit subset as a known
// optimisation) runs before the tile scheduler: see fuse_single_qubit_runs.
#include <chrono>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <numeric>

#include "qs_internal.h"

namespace qs {

int default_tile_bits(int dtype) { return dtype == QS_C128 ? 12 : 13; }

// Per-launch cost coefficients measured on GB300 (ms, ms per byte, ms per counted
// instruction): HBM-bound kernels at the bandwidth they reach (per-gate ~6.4 TB/s,
// permutation ~5.7, dense tensor-core block 3.6 ms per 17.2 GB); a tile pass's per-byte
// term is what a pass with almost no arithmetic costs (complex64 4.4 ms per 17.2 GB;
// double-float fitted on the fused 30-qubit plans, whose passes keep the state in
// double-float form), its per-instruction term the rest of the 30-qubit circuits' time
// (complex64 ~246 ms, double-float ~1084 ms per circuit) over the counted instructions;
// native FP64 at 1.7 DFMA per clock per SM.
qs_cost_model default_cost_model(Policy pol) {
  qs_cost_model m{};
  const double tile_alu = pol == POL_F32 ? 7.0e-11 : (pol == POL_DF ? 4.27e-11 : 1.87e-9);
  const double tile_byte = pol == POL_F32 ? 1.0 / 3.9e9 : (pol == POL_DF ? 1.0 / 5.37e9 : 1.0 / 6.5e9);
  const double c_tile[3] = {0.005, tile_byte, tile_alu};
  const double c_gate[3] = {0.005, 1.0 / 6.4e9, pol == POL_F64 ? 1.87e-9 : 0.0};
  const double c_perm[3] = {0.005, 1.0 / 5.7e9, 0.0};
  const double c_dense[3] = {0.005, 3.6 / 17.18e9, 0.0};
  for (int i = 0; i < 3; i++) {
    m.tile[i] = c_tile[i];
    m.gate[i] = c_gate[i];
    m.permute[i] = c_perm[i];
    m.dense[i] = c_dense[i];
  }
  return m;
}

double step_cost_ms(const qs_cost_model& m, const Step& s) {
  const double* c = nullptr;
  switch (s.kind) {
    case ST_PASS: c = m.tile; break;
    case ST_GATE: c = m.gate; break;
    case ST_PERMUTE: c = m.permute; break;
    case ST_DENSE: c = m.dense; break;
    case ST_RENORM: return s.bytes * m.gate[1] + 2 * m.gate[0];
  }
  return c[0] + c[1] * s.bytes + c[2] * s.alu;
}
// segments of 16 amplitudes (256 bytes) for complex128, 32 (256 bytes) for complex64: swept
// on GB300 with the fused plans (c = 3 / 4 were 2.5 % / 7 % slower on the 30-qubit circuit)
int default_low_bits(int dtype) { return dtype == QS_C128 ? 4 : 5; }

bool normalize_compile_opts(int n, qs_compile_opts* o, std::string* err) {
  auto bad = [&](const char* m) {
    *err = m;
    return false;
  };
  if (o->dtype != QS_C64 && o->dtype != QS_C128) return bad("unknown dtype");
  if (o->mode < QS_MODE_PERGATE || o->mode > QS_MODE_TILE) return bad("unknown mode");
  if (o->flags & ~(QS_FLAG_FULL_RX | QS_FLAG_NO_DENSE | QS_FLAG_NO_FUSE)) return bad("unknown flags");
  if (o->reg_bits < 0 || o->reg_bits > 5) return bad("reg_bits must be in [0, 5]");
  if (o->renorm_every < 0) return bad("renorm_every must be >= 0");
  if (o->tile_bits == 0) o->tile_bits = default_tile_bits(o->dtype);
  if (o->low_bits == 0) o->low_bits = default_low_bits(o->dtype);
  if (o->tile_bits < 1 || (o->mode != QS_MODE_PAPER && o->tile_bits > kMaxTileBits))
    return bad("tile_bits must be in [1, 14] (QS_MODE_PAPER: [1, n])");
  if (o->tile_bits > n) o->tile_bits = n;
  if (o->low_bits > o->tile_bits) o->low_bits = o->tile_bits;
  const int min_low = (o->dtype == QS_C64) ? 1 : 0;   // 16-byte bulk copies
  if (o->low_bits < min_low) o->low_bits = min_low;
  if (o->low_bits > o->tile_bits) return bad("state too small for a tile pass");
  return true;
}

// Gate j depends on an earlier gate i iff they share a qubit on which their action
// classes differ (classes Z and X each commute with themselves, N with nothing).  Per
// qubit, consecutive gates of one commuting class form a group; a gate's immediate
// predecessors on that qubit are the members of the latest group it does not commute with.
std::vector<std::vector<int>> build_dag(const std::vector<HGate>& gates) {
  const int G = (int)gates.size();
  std::vector<std::vector<int>> preds(G);
  struct QState {
    int cls = -1;
    std::vector<int> cur, prev;
  };
  std::vector<QState> qs(kMaxQubits + 1);
  for (int j = 0; j < G; j++) {
    const HGate& g = gates[j];
    for (int t = 0; t < g.nq; t++) {
      QState& s = qs[g.q[t]];
      const int c = g.cls[t];
      if (s.cls >= 0 && c == s.cls && c != CLS_N) {
        preds[j].insert(preds[j].end(), s.prev.begin(), s.prev.end());
        s.cur.push_back(j);
      } else {
        preds[j].insert(preds[j].end(), s.cur.begin(), s.cur.end());
        s.prev.swap(s.cur);
        s.cur.assign(1, j);
        s.cls = c;
      }
    }
    std::sort(preds[j].begin(), preds[j].end());
    preds[j].erase(std::unique(preds[j].begin(), preds[j].end()), preds[j].end());
  }
  return preds;
}

namespace {

// out = a b for row-major 2x2 matrices
void mul2x2(const cd a[4], const cd b[4], cd out[4]) {
  const cd r0 = a[0] * b[0] + a[1] * b[2], r1 = a[0] * b[1] + a[1] * b[3];
  const cd r2 = a[2] * b[0] + a[3] * b[2], r3 = a[2] * b[1] + a[3] * b[3];
  out[0] = r0;
  out[1] = r1;
  out[2] = r2;
  out[3] = r3;
}

bool is_identity(const cd m[4]) { return m[0] == cd(1, 0) && m[1] == cd(0, 0) && m[2] == cd(0, 0) && m[3] == cd(1, 0); }

}  // namespace

// The single-qubit gates acting on one qubit between two multi-qubit gates on that qubit
// commute with every gate in between (those act on other qubits), so they can be applied at
// once, as their product, just before the next multi-qubit gate on the qubit.  Inside a tile
// pass a general single-qubit matrix is applied as diagonal . RX . diagonal (see lower_gate):
// one tangent-form RX update plus two factors of the register phase tables, which are shared
// with the other register qubits.  So a run is fused when it holds two or more non-diagonal
// gates, or a general one (neither RX nor X in form), or consists of diagonal gates only (one
// diagonal factor).  A run whose one non-diagonal gate is an RX or an X is kept as it is.
void fuse_single_qubit_runs(int n, std::vector<HGate>& in, std::vector<HGate>* out, FuseOrigin* origin) {
  out->clear();
  out->reserve(in.size());
  origin->off.assign(1, 0);
  origin->idx.clear();
  origin->idx.reserve(in.size());
  std::vector<std::vector<int>> run(n);
  auto close = [&] { origin->off.push_back((int)origin->idx.size()); };
  auto keep = [&](int i) {   // an input gate as it is (moved: the input is consumed)
    out->push_back(std::move(in[i]));
    origin->idx.push_back(i);
    close();
  };
  auto emit = [&](HGate g, const std::vector<int>& src) {
    out->push_back(std::move(g));
    origin->idx.insert(origin->idx.end(), src.begin(), src.end());
    close();
  };
  auto flush = [&](int q) {
    std::vector<int>& r = run[q];
    if (r.empty()) return;
    int nd = 0;
    bool general = false;
    for (int i : r) {
      if (in[i].cls[0] == CLS_Z) continue;
      nd++;
      const cd* m = in[i].U.data();
      const bool x_form = m[0] == cd(0, 0) && m[3] == cd(0, 0) && m[1] == cd(1, 0) && m[2] == cd(1, 0);
      const bool rx_form = m[0] == m[3] && m[0].imag() == 0.0 && m[1] == m[2] && m[1].real() == 0.0;
      general |= !x_form && !rx_form;
    }
    if (r.size() < 2 || (nd == 1 && !general)) {   // a lone general gate splits at lowering
      for (int i : r) keep(i);
      r.clear();
      return;
    }
    cd U[4] = {1, 0, 0, 1}, t[4];
    for (int i : r) {   // later gates act on the left
      const cd G[4] = {in[i].U[0], in[i].U[1], in[i].U[2], in[i].U[3]};
      mul2x2(G, U, t);
      for (int k = 0; k < 4; k++) U[k] = t[k];
    }
    // the product as separate gates diag, RX, diag: the scheduler may then place the two
    // diagonal factors wherever their phase tables are cheapest
    cd d1[4], rx[4], d2[4];
    if (is_identity(U)) {
      for (int i : r) keep(i);   // an exact identity: keep the gates (rare)
    } else if (U[1] == cd(0, 0) && U[2] == cd(0, 0)) {
      emit(make_1q_gate(q, U), r);
    } else if (euler_split(U, d1, rx, d2)) {
      if (!is_identity(d1)) emit(make_1q_gate(q, d1), {});
      emit(make_1q_gate(q, rx), r);
      if (!is_identity(d2)) emit(make_1q_gate(q, d2), {});
    } else {
      emit(make_1q_gate(q, U), r);
    }
    r.clear();
  };
  for (int i = 0; i < (int)in.size(); i++) {
    const HGate& g = in[i];
    if (g.nq == 1) {
      run[g.q[0]].push_back(i);
      continue;
    }
    for (int t = 0; t < g.nq; t++) flush(g.q[t]);
    keep(i);
  }
  for (int q = 0; q < n; q++) flush(q);
}

namespace {

// Qubits a gate needs inside the tile: those on which it acts non-diagonally; a general
// 2- or k-qubit matrix (applied as a dense block) needs all of its qubits.
bool needs_qubit(const HGate& g, int t) {
  if (g.nq >= 2 && (g.kind == QS_OP_U2 || g.kind == QS_OP_UK)) return true;
  return g.cls[t] != CLS_Z;
}
// storage-bit mask of the qubits the gate needs inside the tile
uint64_t nd_mask(const HGate& g, const std::vector<int>& sigma) {
  uint64_t m = 0;
  for (int t = 0; t < g.nq; t++)
    if (needs_qubit(g, t)) m |= 1ull << sigma[g.q[t]];
  return m;
}

struct Sched {
  const std::vector<HGate>& gates;
  std::vector<std::vector<int>> preds, succs;
  std::vector<int> npred;
  std::vector<char> done;
  std::vector<int> rem;      // remaining gate indices in program order
  int remaining;
  explicit Sched(const std::vector<HGate>& g) : gates(g) {
    const int G = (int)g.size();
    preds = build_dag(g);
    succs.assign(G, {});
    npred.assign(G, 0);
    for (int j = 0; j < G; j++) {
      npred[j] = (int)preds[j].size();
      for (int i : preds[j]) succs[i].push_back(j);
    }
    done.assign(G, 0);
    rem.resize(G);
    std::iota(rem.begin(), rem.end(), 0);
    remaining = G;
  }
  void mark(int v) {
    done[v] = 1;
    remaining--;
    for (int s : succs[v]) npred[s]--;
  }
  void compact() {
    size_t w = 0;
    for (size_t r = 0; r < rem.size(); r++)
      if (!done[rem[r]]) rem[w++] = rem[r];
    rem.resize(w);
  }
  // number of gates one program-order sweep would schedule if every gate whose
  // non-diagonal storage bits lie in `local` (a storage-bit mask) were runnable;
  // `tmp` is scratch of size G.
  template <class Skip>
  int closure(uint64_t local, const std::vector<uint64_t>& ndm, std::vector<char>& tmp, int cap, Skip skip) const {
    int cnt = 0;
    for (int v : rem) {
      bool ok = (ndm[v] & ~local) == 0 && !skip(v);
      if (ok)
        for (int p : preds[v])
          if (!done[p] && !tmp[p]) {
            ok = false;
            break;
          }
      tmp[v] = ok;
      if (ok && ++cnt >= cap) break;
    }
    for (int v : rem) tmp[v] = 0;
    return cnt;
  }
  int closure(uint64_t local, const std::vector<uint64_t>& ndm, std::vector<char>& tmp) const {
    return closure(local, ndm, tmp, 1 << 30, [](int) { return false; });
  }
  // the gates that sweep would schedule, in program order (nothing is marked)
  std::vector<int> collect(uint64_t local, const std::vector<uint64_t>& mask, std::vector<char>& tmp) const {
    std::vector<int> ids;
    for (int v : rem) {
      bool ok = (mask[v] & ~local) == 0;
      if (ok)
        for (int p : preds[v])
          if (!done[p] && !tmp[p]) {
            ok = false;
            break;
          }
      tmp[v] = ok;
      if (ok) ids.push_back(v);
    }
    for (int v : rem) tmp[v] = 0;
    return ids;
  }
};

double gate_bytes(const HGate& g, int n, int store_bytes) {
  // bytes read + written by the per-gate kernel of this gate
  const double S = (double)store_bytes * (double)(1ull << n);
  int fixed = 0;   // bits fixed by controls / phase predicates
  bool diag = true;
  for (int t = 0; t < g.nq; t++)
    if (g.cls[t] != CLS_Z) diag = false;
  if (g.kind == QS_OP_CNOT || g.kind == QS_OP_CU || g.kind == QS_OP_CP || g.kind == QS_OP_CZ) fixed = 1;
  if (g.kind == QS_OP_CZ || g.kind == QS_OP_CP) fixed = 2;
  if (g.nq == 1 && diag && g.U[0] == cd(1, 0)) fixed = 1;   // phase on |1>
  if (g.kind == QS_OP_SWAP) fixed = 1;                        // only |01>,|10> move
  return 2.0 * S / (double)(1ull << fixed);
}

void fill_tile_ctx(LowerCtx* ctx, const int* tpos, int L) {
  for (int b = 0; b < 64; b++) ctx->tile_index[b] = -1;
  for (int k = 0; k < L; k++) ctx->tile_index[tpos[k]] = k;
}

bool emit_pass(int n, int L, int c, const std::vector<int>& tbits_sorted, const std::vector<int>& gate_ids,
               const std::vector<HGate>& gates, const std::vector<int>& sigma, CompileResult* out,
               std::string* err) {
  Step st;
  st.kind = ST_PASS;
  memset(&st.pass, 0, sizeof(st.pass));
  st.pass.L = L;
  st.pass.c = c;
  st.pass.n = n;
  for (int k = 0; k < L; k++) st.pass.tpos[k] = tbits_sorted[k];
  int nn = 0;
  std::vector<char> in(n, 0);
  for (int k = 0; k < L; k++) in[tbits_sorted[k]] = 1;
  for (int b = 0; b < n; b++)
    if (!in[b]) st.pass.npos[nn++] = b;
  LowerCtx ctx;
  ctx.sigma = sigma.data();
  ctx.tile = true;
  fill_tile_ctx(&ctx, st.pass.tpos, L);
  std::vector<DevOp> ops;
  for (int v : gate_ids) {
    if (!lower_gate(gates[v], ctx, out->pool, ops)) {
      *err = "internal: gate not lowerable in its tile pass";
      return false;
    }
  }
  if (ops.empty()) return true;   // identity gates only
  st.pass.K = register_bits(out->store_bytes == 16 ? QS_C128 : QS_C64, L, out->reg_bits);
  build_stages(ops, L, st.pass.K, out, &st.pass.st0, &st.pass.nst);
  bool lite = true;
  for (int k = st.pass.st0; k < st.pass.st0 + st.pass.nst && lite; k++) {
    const StageRec& sr = out->stages[k];
    if (sr.kind != 0) continue;
    for (int i = sr.op0; i < sr.op0 + sr.nops; i++) {
      const int t = out->reg_ops[i].type;
      if (t != OP_RXTM && t != OP_DTAB && t != OP_PHASE && t != OP_RX) lite = false;
    }
  }
  if (lite) st.pass.flags |= kPassLite;
  const int store_bytes = out->store_bytes;
  st.bytes = 2.0 * (double)store_bytes * (double)(1ull << n);
  st.alu = stage_alu_per_amp(*out, st.pass.st0, st.pass.nst) * (double)(1ull << n);
  out->steps.push_back(std::move(st));
  out->stats.n_passes++;
  return true;
}

bool emit_gate(int n, const HGate& g, const std::vector<int>& sigma, int store_bytes, CompileResult* out,
               std::string* err) {
  LowerCtx ctx;
  ctx.sigma = sigma.data();
  ctx.tile = false;
  std::vector<DevOp> ops;
  if (!lower_gate(g, ctx, out->pool, ops)) {
    *err = "internal: gate not lowerable";
    return false;
  }
  for (const DevOp& o : ops) {
    Step st;
    st.kind = ST_GATE;
    st.op = o;
    st.bytes = gate_bytes(g, n, store_bytes);
    st.alu = (op_alu_per_amp(out->pol, o) + (out->pol == POL_DF ? 72.0 : 0.0)) * (double)(1ull << n);
    out->steps.push_back(std::move(st));
  }
  return true;
}

bool emit_permute(int n, const std::vector<int>& sigma, const std::vector<int>& sigma_new, int store_bytes,
                  CompileResult* out) {
  Step st;
  st.kind = ST_PERMUTE;
  st.perm = sigma_new;
  st.src_of.assign(n, 0);
  for (int q = 0; q < n; q++) st.src_of[sigma_new[q]] = sigma[q];
  st.bytes = 2.0 * (double)store_bytes * (double)(1ull << n);
  out->steps.push_back(std::move(st));
  return true;
}

// Fuse gates that act only on storage bits 0..5 into one 64 x 64 unitary (row / column index =
// those bits) and emit it as a dense tensor-core step.
void emit_dense(int n, const std::vector<int>& ids, const std::vector<HGate>& gates, const std::vector<int>& sigma,
                int store_bytes, CompileResult* out) {
  constexpr int D = 64;
  std::vector<cd> M(D * D, cd(0, 0));
  for (int i = 0; i < D; i++) M[i * D + i] = 1.0;
  std::vector<cd> x(D), y(D);
  for (int v : ids) {   // M <- G M, one column at a time
    const HGate& g = gates[v];
    const int k = g.nq, dk = 1 << k;
    int pos[6];
    uint32_t mask = 0;
    for (int t = 0; t < k; t++) {
      pos[t] = sigma[g.q[t]];
      mask |= 1u << pos[t];
    }
    for (int col = 0; col < D; col++) {
      for (int i = 0; i < D; i++) x[i] = M[i * D + col];
      y = x;
      for (int base = 0; base < D; base++) {
        if (base & mask) continue;
        for (int r = 0; r < dk; r++) {
          int ir = base;
          for (int t = 0; t < k; t++)
            if ((r >> t) & 1) ir |= 1 << pos[t];
          cd acc(0, 0);
          for (int c = 0; c < dk; c++) {
            int ic = base;
            for (int t = 0; t < k; t++)
              if ((c >> t) & 1) ic |= 1 << pos[t];
            acc += g.U[r * dk + c] * x[ic];
          }
          y[ir] = acc;
        }
      }
      for (int i = 0; i < D; i++) M[i * D + col] = y[i];
    }
  }
  Step st;
  st.kind = ST_DENSE;
  st.dense_idx = (int32_t)(out->dense_u.size() / (D * D));
  st.bytes = 2.0 * (double)store_bytes * (double)(1ull << n);
  out->dense_u.insert(out->dense_u.end(), M.begin(), M.end());
  std::vector<double> flat(2 * D * D);
  for (int i = 0; i < D * D; i++) {
    flat[2 * i] = M[i].real();
    flat[2 * i + 1] = M[i].imag();
  }
  const int bits[6] = {0, 1, 2, 3, 4, 5};
  const size_t w0 = out->dense_w.size();
  out->dense_w.resize(w0 + kDenseWFloats);
  dense_mma_weights(flat.data(), 6, bits, out->dense_w.data() + w0);
  out->steps.push_back(std::move(st));
  out->stats.n_dense++;
}

// ---------------------------------------------------------------------------------------
// QS_MODE_PAPER: Algorithm 1 with m = L local storage positions.
// Readings (as in the tests' reference): the sweep visits remaining gates in program order
// and a removed gate unblocks its successors later in the same sweep; candidates
// sigma o (l g) run over local qubits l then global qubits g in ascending qubit order; the
// score is the number of gates the next sweep would schedule under the candidate
// ("closure", default) or the number of frontier gates it makes local with the count of
// all remaining gates it makes local as tie-break ("frontier"); the first best candidate
// wins; with no positive score the first frontier gate runs non-locally.
bool compile_paper(int n, const std::vector<HGate>& gates, std::vector<int> sigma, const qs_compile_opts& o,
                   int store_bytes, CompileResult* out, std::string* err) {
  const int L = o.tile_bits;
  const int m = L;
  const int G = (int)gates.size();
  Sched S(gates);
  std::vector<char> tmp(G, 0);
  std::vector<int> run;   // consecutive local gates -> one tile pass over storage bits [0, L)
  std::vector<int> tpos(L);
  std::iota(tpos.begin(), tpos.end(), 0);
  auto flush = [&]() -> bool {
    if (run.empty()) return true;
    bool ok = true;
    if (L <= kMaxTileBits) {
      ok = emit_pass(n, L, std::min(o.low_bits, L), tpos, run, gates, sigma, out, err);
    } else {   // more local qubits than a tile holds: the run executes gate by gate
      for (int v : run) {
        ok = ok && emit_gate(n, gates[v], sigma, store_bytes, out, err);
        out->stats.n_pergate++;
      }
    }
    run.clear();
    return ok;
  };
  // logical-qubit masks of the non-diagonal qubits of every gate
  std::vector<uint64_t> ndq(G, 0);
  for (int v = 0; v < G; v++)
    for (int t = 0; t < gates[v].nq; t++)
      if (needs_qubit(gates[v], t)) ndq[v] |= 1ull << gates[v].q[t];
  auto local_mask = [&](const std::vector<int>& sg) {
    uint64_t lm = 0;
    for (int q = 0; q < n; q++)
      if (sg[q] < m) lm |= 1ull << q;
    return lm;
  };
  while (S.remaining) {
    // scheduling sweep: every remaining gate that is local under sigma, in program order
    const uint64_t lm = local_mask(sigma);
    for (int v : S.rem) {
      if (S.done[v] || S.npred[v] != 0 || (ndq[v] & ~lm)) continue;
      S.mark(v);
      out->trace.push_back({0, v});
      run.push_back(v);
      if (o.max_ops > 0 && (int)run.size() >= o.max_ops && !flush()) return false;
    }
    S.compact();
    if (!S.remaining) break;
    // score every local<->global transposition
    std::vector<int> loc, glo;
    for (int q = 0; q < n; q++) (sigma[q] < m ? loc : glo).push_back(q);
    int best_l = -1, best_g = -1;
    long best0 = 0, best1 = -1;
    bool have = false;
    for (int l : loc)
      for (int g : glo) {
        const uint64_t lm2 = (lm & ~(1ull << l)) | (1ull << g);
        long f, a = 0;
        if (o.scoring == 0) {
          f = S.closure(lm2, ndq, tmp);
        } else {
          f = 0;
          for (int v : S.rem) {
            if (ndq[v] & ~lm2) continue;
            a++;
            if (S.npred[v] == 0) f++;
          }
        }
        if (!have || f > best0 || (o.scoring != 0 && f == best0 && a > best1)) {
          have = true;
          best0 = f;
          best1 = a;
          best_l = l;
          best_g = g;
        }
      }
    // apply the best transposition, or run the first frontier gate non-locally
    if (have && best0 > 0) {
      const size_t nsteps = out->steps.size();
      if (!flush()) return false;
      std::vector<int> sg = sigma;
      std::swap(sg[best_l], sg[best_g]);
      const int pl = sigma[best_l], pg = sigma[best_g];
      // PermuteQubits on the store of the tile pass just flushed (it reads under sigma and
      // writes under sigma'): exchanging storage bits pl and pg moves whole 2^c-element
      // segments as long as pl >= c, so it costs no extra pass; otherwise a permutation kernel
      Step* last = out->steps.size() > nsteps ? &out->steps.back() : nullptr;
      if (last && last->kind == ST_PASS && last->pass.swap_a == last->pass.swap_b && pl >= last->pass.c) {
        last->pass.swap_a = pl;
        last->pass.swap_b = pg;
        last->perm = sg;
      } else {
        emit_permute(n, sigma, sg, store_bytes, out);
        out->stats.n_permute_kernels++;
      }
      out->stats.n_permutes++;
      out->trace.push_back({2, best_l * 64 + best_g});
      sigma = sg;
    } else {
      int v = -1;
      for (int u : S.rem)
        if (S.npred[u] == 0) {
          v = u;
          break;
        }
      if (v < 0) {
        *err = "internal: no frontier gate";
        return false;
      }
      if (!flush()) return false;
      S.mark(v);
      S.compact();
      out->trace.push_back({1, v});
      if (!emit_gate(n, gates[v], sigma, store_bytes, out, err)) return false;
      out->stats.n_pergate++;
      out->stats.n_comm_gates++;
    }
  }
  if (!flush()) return false;
  out->sigma_final = sigma;
  return true;
}

// ---------------------------------------------------------------------------------------
// QS_MODE_TILE: every pass picks its own set of L storage bits (the c lowest always in),
// greedily: starting from the c low bits, add the bit whose inclusion lets one program-order
// sweep schedule the most gates (ties: the bit most wanted by frontier gates, then the
// lowest bit).  The pass then runs that sweep.
// origin (may be null): the input gates each entry of `gates` stands for (gate fusion)
bool compile_tile(int n, const std::vector<HGate>& gates, const std::vector<int>& sigma, const qs_compile_opts& o,
                  int store_bytes, CompileResult* out, std::string* err, const FuseOrigin* origin = nullptr) {
  const int L = std::min(o.tile_bits, n);
  const int c = std::min(o.low_bits, L);
  const int G = (int)gates.size();
  Sched S(gates);
  std::vector<uint64_t> ndm(G);
  for (int v = 0; v < G; v++) ndm[v] = nd_mask(gates[v], sigma);
  std::vector<char> tmp(G, 0);
  const uint64_t low = (c >= 64) ? ~0ull : ((1ull << c) - 1);
  // fully diagonal gates none of whose qubits is in the tile are deferred to a pass that
  // holds one of them (there they merge into a register phase table); only gates acting
  // non-diagonally on those qubits depend on them, and those cannot run in this pass anyway
  std::vector<char> allz(G, 0);
  std::vector<uint64_t> qmask(G, 0);
  int nondiag_left = 0;
  for (int v = 0; v < G; v++) {
    bool z = true;
    for (int t = 0; t < gates[v].nq; t++) {
      qmask[v] |= 1ull << sigma[gates[v].q[t]];
      if (gates[v].cls[t] != CLS_Z) z = false;
    }
    allz[v] = z;
    if (!z) nondiag_left++;
  }
  auto deferred = [&](int v, uint64_t T) { return allz[v] && (qmask[v] & T) == 0 && nondiag_left > 0; };
  std::vector<uint64_t> okm(G, 0);   // candidate-bit masks of the pass search
  for (int v = 0; v < G; v++)
    if (__builtin_popcountll(ndm[v] | low) > L) {
      const int g0 = (origin && origin->count(v)) ? origin->idx[origin->off[v]] : v;
      *err = "gate " + std::to_string(g0) + " needs more qubits than a tile holds";
      return false;
    }
  // dense blocks on the tensor cores (complex64): every gate's full storage-bit set
  const bool dense_ok = out->pol == POL_F32 && !(o.flags & QS_FLAG_NO_DENSE) && n >= dense_mma_min_qubits();
  std::vector<uint64_t> allq(G, 0);
  std::vector<double> wsave(G, 0.0);
  double t_dense = 0;
  if (dense_ok) {
    const double S2 = 2.0 * (double)store_bytes * (double)(1ull << n);
    t_dense = out->cost.dense[0] + out->cost.dense[1] * S2;
    for (int v = 0; v < G; v++) {
      for (int t = 0; t < gates[v].nq; t++) allq[v] |= 1ull << sigma[gates[v].q[t]];
      // tile-pass time the gate would cost: its arithmetic at the tile class's rate
      wsave[v] = out->cost.tile[2] * gate_tile_alu_per_amp(out->pol, gates[v]) * (double)(1ull << n);
    }
  }
  while (S.remaining) {
    if (dense_ok) {
      // the gates ready on storage bits 0..5 alone: one dense block if the model says it
      // is cheaper than leaving them to the tile passes
      std::vector<int> ids = S.collect(63ull, allq, tmp);
      double save = 0;
      for (int v : ids) save += wsave[v];
      if (!ids.empty() && save > t_dense) {
        for (int v : ids) {
          S.mark(v);
          bool z = true;
          for (int t = 0; t < gates[v].nq; t++) z &= gates[v].cls[t] == CLS_Z;
          if (!z) nondiag_left--;
        }
        S.compact();
        out->trace.push_back({5, (int)ids.size()});
        for (int v : ids) out->trace.push_back({0, v});
        emit_dense(n, ids, gates, sigma, store_bytes, out);
        continue;
      }
    }
    uint64_t T = low;
    int nt = c;
    // demand: how many frontier gates need each bit
    std::vector<int> demand(n, 0);
    for (int v : S.rem)
      if (S.npred[v] == 0)
        for (int b = 0; b < n; b++)
          if ((ndm[v] >> b) & 1) demand[b]++;
    while (nt < L) {
      // one program-order sweep scores every candidate bit b at once: okm[v] has bit b set
      // iff gate v would be scheduled in a pass over T | b (its non-diagonal bits covered,
      // not deferred, every unfinished predecessor scheduled as well)
      const uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1);
      const uint64_t cand = all & ~T;
      int score[64] = {0};
      for (int v : S.rem) {
        const uint64_t miss = ndm[v] & ~T;
        uint64_t m = (miss == 0) ? cand : ((miss & (miss - 1)) == 0 ? (miss & cand) : 0ull);
        if (m && allz[v] && nondiag_left > 0 && !(qmask[v] & T)) m &= qmask[v];   // deferred unless b is one of its bits
        for (int p : S.preds[v]) {
          if (!m) break;
          if (!S.done[p]) m &= okm[p];
        }
        okm[v] = m;
        // a gate that runs under every candidate adds the same to every score: skipped
        if (m != cand)
          for (uint64_t mm = m; mm; mm &= mm - 1) score[__builtin_ctzll(mm)]++;
      }
      int best_b = -1, best_s = -1, best_d = -1;
      for (int b = 0; b < n; b++) {
        if ((T >> b) & 1) continue;
        if (score[b] > best_s || (score[b] == best_s && demand[b] > best_d)) {
          best_s = score[b];
          best_d = demand[b];
          best_b = b;
        }
      }
      if (best_b < 0) break;
      T |= 1ull << best_b;
      nt++;
    }
    // the sweep of this pass
    std::vector<int> ids;
    for (int v : S.rem) {
      if (S.done[v] || S.npred[v] != 0 || (ndm[v] & ~T) || deferred(v, T)) continue;
      S.mark(v);
      if (!allz[v]) nondiag_left--;
      ids.push_back(v);
      if (o.max_ops > 0 && (int)ids.size() >= o.max_ops) break;
    }
    S.compact();
    if (ids.empty()) {
      *err = "internal: tile pass scheduled no gate (a gate needs more than L - low_bits tile bits)";
      return false;
    }
    std::vector<int> tb;
    for (int b = 0; b < n; b++)
      if ((T >> b) & 1) tb.push_back(b);
    out->trace.push_back({3, (int)(T & 0x7FFFFFFFull)});
    out->trace.push_back({4, (int)(T >> 31)});
    for (int v : ids) out->trace.push_back({0, v});
    if (!emit_pass(n, (int)tb.size(), c, tb, ids, gates, sigma, out, err)) return false;
  }
  out->sigma_final = sigma;
  return true;
}

// Between two tile passes that follow one another (permutations in between move 16-byte
// elements unchanged) the state stays in the double-float storage form, so that those
// passes skip the binary64 split on load and the join on store; the plan's first pass reads
// binary64, and a pass followed by anything else (a per-gate kernel, a renormalisation, the
// end of the plan) writes binary64.  A pass without stages only moves data (a permutation
// fused into its store) and keeps the form it reads.  The counted conversion work of a pass
// drops accordingly: split 36 and join 36 instruction equivalents per amplitude, the
// double-float store's normalisation 12.
void set_double_float_storage(int n, CompileResult* out) {
  const size_t S = out->steps.size();
  auto real_pass = [&](size_t i) { return out->steps[i].kind == ST_PASS && out->steps[i].pass.nst > 0; };
  bool fmt_df = false;
  for (size_t i = 0; i < S; i++) {
    Step& s = out->steps[i];
    if (s.kind != ST_PASS) continue;
    s.pass.flags &= ~(kPassInDF | kPassOutDF);
    if (!real_pass(i)) {
      if (fmt_df) s.pass.flags |= kPassInDF | kPassOutDF;
      continue;
    }
    bool next_df = false;
    for (size_t j = i + 1; j < S; j++) {
      if (out->steps[j].kind == ST_PERMUTE || (out->steps[j].kind == ST_PASS && !real_pass(j))) continue;
      next_df = real_pass(j);
      break;
    }
    const double amps = (double)(1ull << n);
    if (fmt_df) {
      s.pass.flags |= kPassInDF;
      s.alu -= 36.0 * amps;
    }
    if (next_df) {
      s.pass.flags |= kPassOutDF;
      s.alu -= 24.0 * amps;
    }
    fmt_df = next_df;
  }
}

}  // namespace

bool compile_circuit(int n, std::vector<HGate> gates, const std::vector<int>& sigma0,
                     const qs_compile_opts& o, CompileResult* out, std::string* err) {
  auto t0 = std::chrono::steady_clock::now();
  const int store_bytes = (o.dtype == QS_C128) ? 16 : 8;
  out->store_bytes = store_bytes;
  out->reg_bits = o.reg_bits;
  out->full_rx = (o.flags & QS_FLAG_FULL_RX) != 0;
  out->pol = (o.dtype == QS_C64) ? POL_F32 : (o.arith == QS_ARITH_F64 ? POL_F64 : POL_DF);
  out->cost = o.cost ? *o.cost : default_cost_model(out->pol);
  out->stats = qs_plan_stats{};
  out->stats.n_gates = (int64_t)gates.size();
  bool ok = true;
  bool has_relabel = false;
  for (const HGate& g : gates) has_relabel |= g.kind == QS_OP_RELABEL;
  if (has_relabel && o.mode != QS_MODE_PERGATE) {
    *err = "RELABEL (Emulated-SWAP) ops need QS_MODE_PERGATE";
    return false;
  }
  if (o.mode == QS_MODE_PERGATE) {
    std::vector<int> sigma = sigma0;
    for (const HGate& g : gates) {
      if (g.kind == QS_OP_RELABEL) {   // storage positions change hands, no data moves
        std::swap(sigma[g.q[0]], sigma[g.q[1]]);
        continue;
      }
      if (!emit_gate(n, g, sigma, store_bytes, out, err)) return false;
      out->stats.n_pergate++;
    }
    out->sigma_final = sigma;
  } else if (o.mode == QS_MODE_PAPER) {
    ok = compile_paper(n, gates, sigma0, o, store_bytes, out, err);
  } else if (o.mode == QS_MODE_TILE) {
    if (o.flags & QS_FLAG_NO_FUSE) {
      ok = compile_tile(n, gates, sigma0, o, store_bytes, out, err);
    } else {
      std::vector<HGate> fused;
      FuseOrigin origin;
      fuse_single_qubit_runs(n, gates, &fused, &origin);   // consumes gates
      ok = compile_tile(n, fused, sigma0, o, store_bytes, out, err, &origin);
      for (size_t i = 0; i < fused.size(); i++)
        if (origin.count(i) >= 2) out->stats.n_fused += origin.count(i);
      if (ok) {   // the trace names input gates: a fused gate lists the gates it stands for
        std::vector<std::pair<int, int>> tr;
        tr.reserve(out->trace.size());
        for (size_t i = 0; i < out->trace.size(); i++) {
          const auto& e = out->trace[i];
          if (e.first == 0) {
            for (int k = origin.off[e.second]; k < origin.off[e.second + 1]; k++) tr.push_back({0, origin.idx[k]});
          } else if (e.first == 5) {   // dense block over the next e.second (fused) gates
            int cnt = 0;
            for (int k = 1; k <= e.second && i + k < out->trace.size(); k++)
              cnt += origin.count(out->trace[i + k].second);
            tr.push_back({5, cnt});
          } else {
            tr.push_back(e);
          }
        }
        out->trace.swap(tr);
      }
    }
  } else {
    *err = "unknown compile mode";
    return false;
  }
  if (!ok) return false;
  if (o.renorm_every > 0) {   // FP64 norm (read) + scaling (read + write) after every R kernels
    std::vector<Step> with;
    int since = 0;
    for (Step& s : out->steps) {
      with.push_back(std::move(s));
      if (++since == o.renorm_every) {
        Step r;
        r.kind = ST_RENORM;
        r.bytes = 3.0 * (double)store_bytes * (double)(1ull << n);
        with.push_back(std::move(r));
        since = 0;
      }
    }
    out->steps = std::move(with);
  }
  if (out->pol == POL_DF) set_double_float_storage(n, out);
  double bytes = 0, alu = 0;
  for (const Step& s : out->steps) {
    bytes += s.bytes;
    alu += s.alu;
  }
  out->stats.hbm_bytes = bytes;
  out->stats.alu_instr = alu;
  double pred = 0;
  for (const Step& s : out->steps) pred += step_cost_ms(out->cost, s);
  out->stats.predicted_ms = pred;
  out->stats.compile_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return true;
}

}  // namespace qs
