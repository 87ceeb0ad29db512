// Stage builder for tile passes: groups a pass's ops so that most of them run on
// amplitudes held in registers.
//
// In a register stage every thread holds 2^K amplitudes of the tile -- those that differ
// only in the stage's K register bits R -- and applies, in program order, every op whose
// non-diagonal target bits lie in R; diagonal ops (phases, controls) apply to any bit.  A
// stage costs one shared-memory round trip of the tile instead of one per gate.  R is
// chosen like the pass's own bit set: greedily add the tile bit that lets one program-order
// sweep schedule the most ops (ties: the bit the earliest ready op needs, then the lowest
// bit).  Dense k-qubit blocks and SWAPs run as shared-memory stages.
#include <string.h>

#include <algorithm>
#include <vector>

#include <cmath>

#include "qs_internal.h"

namespace qs {

namespace {

struct OpInfo {
  uint32_t need = 0;      // tile bits that must be in registers (non-diagonal targets)
  uint32_t tbits = 0;     // every tile bit the op touches
  bool smem_only = false; // dense / swap
  int nb = 0;
  int bit[8];
  int cls[8];
};

OpInfo classify_op(const DevOp& o) {
  OpInfo in;
  auto add = [&](int b, int c) {
    in.bit[in.nb] = b;
    in.cls[in.nb] = c;
    in.nb++;
    in.tbits |= 1u << b;
  };
  const uint32_t cm = (uint32_t)o.cmask;
  for (int b = 0; b < 32; b++)
    if ((cm >> b) & 1u) add(b, CLS_Z);
  // register-stage U1 / RX carry at most one control, which becomes a 4x4 block
  if ((o.type == OP_U1 || o.type == OP_RX) && __builtin_popcount(cm) >= 2) in.smem_only = true;
  switch (o.type) {
    case OP_U1: add(o.k0, CLS_N); in.need = 1u << o.k0; break;
    case OP_RX:
    case OP_X: add(o.k0, CLS_X); in.need = 1u << o.k0; break;
    case OP_DIAG: if (o.k0 >= 0) add(o.k0, CLS_Z); break;
    case OP_PHASE: break;
    case OP_U2: add(o.k0, CLS_N); add(o.k1, CLS_N); in.need = (1u << o.k0) | (1u << o.k1); break;
    case OP_SWAP: add(o.k0, CLS_N); add(o.k1, CLS_N); in.smem_only = true; break;
    case OP_DENSE:
      for (int t = 0; t < o.nk; t++) add(o.kq[t], CLS_N);
      in.smem_only = true;
      break;
    default: in.smem_only = true; break;
  }
  return in;
}

bool is_diag(const RegOp& r) { return r.type == OP_DIAG || r.type == OP_PHASE; }

// register slots a diagonal op reads (its own slot and its slot controls)
uint32_t diag_slots(const RegOp& r) {
  uint32_t m = r.csl;
  if (r.type == OP_DIAG && r.s0 >= 0) m |= 1u << r.s0;
  return m;
}
uint32_t target_slots(const RegOp& r) {
  uint32_t m = 0;
  if (r.s0 >= 0) m |= 1u << r.s0;
  if (r.type == OP_U2 && r.s1 >= 0) m |= 1u << r.s1;
  return m;
}
// a factor that depends on the register slots only (no group or block dependence)
bool slot_only(const RegOp& r) {
  if (!is_diag(r) || r.cot != 0 || r.gmask != 0) return false;
  if (r.type == OP_DIAG) return r.s0 >= 0;
  return true;
}

uint32_t ctrl_slots(const RegOp& r) { return r.csl; }

// Two register ops must keep their order iff one changes a slot the other reads: a
// non-diagonal op changes its target slots; every op reads its targets and slot controls.
// Reorder a stage's ops (a valid linear extension of those conflicts) so that diagonal ops
// form long runs -- repeatedly emit every ready diagonal op, then every ready non-diagonal
// one -- and replace the slot-only diagonal factors of each run by one table op:
// entry j of a 2^K-entry table is the product of the run's factors at register index j
// (computed on the host in FP64).
// Working arrays of merge_diagonals, kept per thread: the function runs once per register
// stage (tens of thousands of times for a large batch of small circuits), and allocating
// them on every call cost more than the merge itself.
struct MergeScratch {
  std::vector<std::pair<int, int>> edges;   // (from, to)
  std::vector<int> indeg, seen, soff, succ, fill, pick;
  std::vector<int> readers[32];
  std::vector<int> ready[2];   // [0] non-diagonal, [1] diagonal
  std::vector<RegOp> ord, out, fac, rest, gen;
};

void merge_diagonals(std::vector<RegOp>& rl, int K, Pool& pool) {
  thread_local MergeScratch ws;
  const int N = (int)rl.size();
  // conflict edges from per-slot state: op j follows the last op that wrote a slot j reads
  // or writes, and every op that read a slot j writes since that slot's last write (the
  // other conflicts follow by transitivity); O(N K) instead of testing every pair
  std::vector<std::pair<int, int>>& edges = ws.edges;
  edges.clear();
  std::vector<int>& indeg = ws.indeg;
  std::vector<int>& seen = ws.seen;
  indeg.assign(N, 0);
  seen.assign(N, -1);
  int last_w[32];
  std::vector<int>* readers = ws.readers;
  for (int b = 0; b < 32; b++) {
    last_w[b] = -1;
    readers[b].clear();
  }
  auto edge = [&](int i, int j) {
    if (seen[i] == j) return;
    seen[i] = j;
    edges.push_back({i, j});
    indeg[j]++;
  };
  for (int j = 0; j < N; j++) {
    const RegOp& r = rl[j];
    const uint32_t w = is_diag(r) ? 0u : target_slots(r);
    const uint32_t rd = (is_diag(r) ? diag_slots(r) : target_slots(r)) | ctrl_slots(r);
    for (uint32_t m = rd | w; m; m &= m - 1) {
      const int b = __builtin_ctz(m);
      if (last_w[b] >= 0) edge(last_w[b], j);
    }
    for (uint32_t m = w; m; m &= m - 1)
      for (int i : readers[__builtin_ctz(m)]) edge(i, j);
    for (uint32_t m = rd & ~w; m; m &= m - 1) readers[__builtin_ctz(m)].push_back(j);
    for (uint32_t m = w; m; m &= m - 1) {
      const int b = __builtin_ctz(m);
      last_w[b] = j;
      readers[b].clear();
    }
  }
  // successors in one array (counting sort of the edges by source)
  std::vector<int>& soff = ws.soff;
  std::vector<int>& succ = ws.succ;
  std::vector<int>& fill = ws.fill;
  soff.assign(N + 1, 0);
  succ.resize(edges.size());
  for (const auto& e : edges) soff[e.first + 1]++;
  for (int j = 0; j < N; j++) soff[j + 1] += soff[j];
  fill.assign(soff.begin(), soff.end() - 1);
  for (const auto& e : edges) succ[fill[e.first]++] = e.second;
  // rounds: every op ready at the round's start of the wanted kind (diagonal, then not), in
  // program order; ops of one round never depend on each other
  std::vector<RegOp>& ord = ws.ord;
  ord.clear();
  ord.reserve(N);
  std::vector<int>* ready = ws.ready;
  ready[0].clear();
  ready[1].clear();
  for (int j = 0; j < N; j++)
    if (indeg[j] == 0) ready[is_diag(rl[j]) ? 1 : 0].push_back(j);
  int left = N;
  bool want_diag = true;
  std::vector<int>& pick = ws.pick;
  while (left > 0) {
    pick.clear();
    pick.swap(ready[want_diag ? 1 : 0]);
    std::sort(pick.begin(), pick.end());
    for (int j : pick) {
      ord.push_back(rl[j]);
      left--;
    }
    for (int j : pick)
      for (int q = soff[j]; q < soff[j + 1]; q++) {
        const int k = succ[q];
        if (--indeg[k] == 0) ready[is_diag(rl[k]) ? 1 : 0].push_back(k);
      }
    want_diag = !want_diag;
  }
  rl.swap(ord);
  std::vector<RegOp>& out = ws.out;
  std::vector<RegOp>& fac = ws.fac;
  std::vector<RegOp>& rest = ws.rest;
  std::vector<RegOp>& gen = ws.gen;
  out.clear();
  out.reserve(rl.size());
  size_t i = 0;
  const int D = 1 << K;
  while (i < rl.size()) {
    if (!is_diag(rl[i])) {
      out.push_back(rl[i++]);
      continue;
    }
    size_t e = i;
    while (e < rl.size() && is_diag(rl[e])) e++;
    fac.clear();
    rest.clear();
    for (size_t k = i; k < e; k++) (slot_only(rl[k]) ? fac : rest).push_back(rl[k]);
    if (!fac.empty()) {   // even a single slot factor: a table multiply avoids per-element selects
      // entry j = product of the run's factors at register index j, divided by entry 0; an
      // entry whose factors all equal their values at index 0 is exactly 1 and skipped (it is
      // outside the mask), and entry 0's value (a phase of the whole tile) is kept after the
      // table for the pass-level fold
      cd tab[32];
      for (int j = 0; j < D; j++) tab[j] = cd(1, 0);
      uint32_t mask = 0;
      // factors on one slot (a diagonal on the slot, a phase where only that slot's bit is
      // set) multiply into one pair (value at bit 0, value at bit 1) first, so that the table
      // costs one pass per slot instead of one per factor
      cd sd[32][2];
      uint32_t used = 0;
      gen.clear();
      for (const RegOp& r : fac) {
        int sl = -1;
        cd d0(1, 0), d1(1, 0);
        if (r.type == OP_DIAG && r.csl == 0 && r.s0 >= 0) {
          sl = r.s0;
          d0 = cd(pool.f64[2 * r.mat], pool.f64[2 * r.mat + 1]);
          d1 = cd(pool.f64[2 * (r.mat + 1)], pool.f64[2 * (r.mat + 1) + 1]);
        } else if (r.type == OP_PHASE && __builtin_popcount(r.csl) == 1) {
          sl = __builtin_ctz(r.csl);
          d1 = r.neg ? cd(-1, 0) : cd(pool.f64[2 * r.mat], pool.f64[2 * r.mat + 1]);
        }
        if (sl < 0) {
          gen.push_back(r);
          continue;
        }
        if (!((used >> sl) & 1u)) {
          sd[sl][0] = sd[sl][1] = cd(1, 0);
          used |= 1u << sl;
        }
        sd[sl][0] *= d0;
        sd[sl][1] *= d1;
      }
      for (uint32_t u = used; u; u &= u - 1) {
        const int sl = __builtin_ctz(u);
        for (int j = 0; j < D; j++) tab[j] *= sd[sl][(j >> sl) & 1];
        if (sd[sl][0] != sd[sl][1])
          for (int j = 0; j < D; j++)
            if ((j >> sl) & 1) mask |= 1u << j;
      }
      for (const RegOp& r : gen) {
        // this factor's value at register index j (1 where its slot controls are not all set)
        auto fval = [&](int j) -> cd {
          if (((uint32_t)j & r.csl) != r.csl) return cd(1, 0);
          if (r.type == OP_DIAG) {
            const int m = r.mat + (((j >> r.s0) & 1) ? 1 : 0);
            return cd(pool.f64[2 * m], pool.f64[2 * m + 1]);
          }
          return r.neg ? cd(-1, 0) : cd(pool.f64[2 * r.mat], pool.f64[2 * r.mat + 1]);
        };
        const cd f0 = fval(0);
        for (int j = 0; j < D; j++) {
          if (((uint32_t)j & r.csl) != r.csl) continue;
          const cd f = fval(j);
          tab[j] *= f;
          if (f != f0) mask |= 1u << j;
        }
      }
      // a phase without slot controls multiplies every entry alike: it only changes entry 0
      const cd t0 = tab[0];
      RegOp t;
      memset(&t, 0, sizeof(t));
      t.type = OP_DTAB;
      t.s0 = t.s1 = t.tb = -1;
      t.gbit = -1;
      t.csl = mask;
      if (pool.entries() & 1) pool.add(cd(0, 0));   // tables start at an even entry (16-byte aligned)
      t.mat = (int)pool.entries();
      for (int j = 0; j < D; j++) pool.add(((mask >> j) & 1u) ? tab[j] / t0 : cd(1, 0));
      pool.add(t0);
      out.push_back(t);
    } else {
      rest.insert(rest.begin(), fac.begin(), fac.end());
    }
    out.insert(out.end(), rest.begin(), rest.end());
    i = e;
  }
  rl.swap(out);
  if (N > (1 << 16)) ws = MergeScratch();   // keep no arrays of an unusually large stage
}

}  // namespace

// Pass-level scalars.  Every uncontrolled register-stage RX may run in tangent form,
// (I - i t X) or (t I - i X) with |t| <= 1, dropping a real factor cos or sin; every phase
// table dropped its entry-0 phase.  Both are scalars on the whole tile, so they commute with
// every op of the pass and may be applied anywhere in it.  A tangent step multiplies every
// amplitude by 1 / |dropped factor| (up to sqrt 2), so a pass of hundreds of them would leave
// the floating-point range; the dropped factors are therefore absorbed in segments: when the
// current segment's growth would pass 2^kSegBits, the next uncontrolled RX keeps the full
// form and also multiplies by the segment's factors, which brings the magnitudes back.  The
// last segment's factors and the table phases multiply the first table of the pass (all of
// its entries then get multiplied), or, in a pass without tables, the pass's first RX, which
// keeps the full form; magnitudes stay within 2^(+-kSegBits) of the unit-norm state.
void fold_pass_factors(CompileResult* out, int st0, int nst, int K) {
  constexpr double kSegBits = 24.0;
  Pool& pool = out->pool;
  const int Dn = 1 << K;   // table entries
  std::vector<int> tabs, rxs;   // indices into out->reg_ops, in execution order
  for (int k = st0; k < st0 + nst; k++) {
    const StageRec& st = out->stages[k];
    if (st.kind != 0) continue;
    for (int i = st.op0; i < st.op0 + st.nops; i++) {
      const RegOp& r = out->reg_ops[i];
      if (r.type == OP_DTAB) tabs.push_back(i);
      else if (r.type == OP_RX && r.csl == 0 && r.cot == 0 && r.gmask == 0) rxs.push_back(i);
    }
  }
  cd factor(1, 0);
  for (int i : tabs) {
    const RegOp& r = out->reg_ops[i];
    factor *= cd(pool.f64[2 * (size_t)(r.mat + Dn)], pool.f64[2 * (size_t)(r.mat + Dn) + 1]);
  }
  const size_t first_rx_kept = (!tabs.empty() || rxs.empty()) ? rxs.size() : 0;   // index in rxs kept full
  double scale = 1.0, grow = 0.0;   // the current segment's dropped factors and their log2 growth
  for (size_t q = 0; q < rxs.size(); q++) {
    if (out->full_rx || q == first_rx_kept) continue;
    RegOp& r = out->reg_ops[rxs[q]];
    double* e = &pool.f64[2 * (size_t)r.mat];
    const double c = e[0], sn = e[1];
    const double g = -std::log2(std::max(std::fabs(c), std::fabs(sn)));
    if (grow + g > kSegBits) {   // full form, closing the segment
      e[0] *= scale;
      e[1] *= scale;
      scale = 1.0;
      grow = 0.0;
      continue;
    }
    grow += g;
    r.type = OP_RXT;
    if (std::fabs(c) >= std::fabs(sn)) {
      r.s1 = 0;
      e[0] = sn / c;
      scale *= c;
    } else {
      r.s1 = 1;
      e[0] = c / sn;
      scale *= sn;
    }
    e[1] = 0.0;
  }
  factor *= scale;
  if (!tabs.empty()) {
    RegOp& r = out->reg_ops[tabs[0]];
    for (int j = 0; j < Dn; j++) {
      const cd v = cd(pool.f64[2 * (size_t)(r.mat + j)], pool.f64[2 * (size_t)(r.mat + j) + 1]) * factor;
      pool.f64[2 * (size_t)(r.mat + j)] = v.real();
      pool.f64[2 * (size_t)(r.mat + j) + 1] = v.imag();
    }
    r.csl = (Dn >= 32) ? 0xFFFFFFFFu : ((1u << Dn) - 1u);
  } else if (!rxs.empty() && first_rx_kept < rxs.size()) {
    double* e = &pool.f64[2 * (size_t)out->reg_ops[rxs[first_rx_kept]].mat];
    e[0] *= factor.real();
    e[1] *= factor.real();
  }
}

// Runs of tangent-form RX on distinct register slots (they commute) become one op: one
// decode for up to K rotations.  A single rotation becomes such an op too, since the merged
// op has the kernels' fast path.  Rebuilds the pass's register-op range in place.
void merge_rxt_runs(CompileResult* out, int st0, int nst) {
  int first = -1;
  for (int k = st0; k < st0 + nst; k++)
    if (out->stages[k].kind == 0) {
      first = out->stages[k].op0;
      break;
    }
  if (first < 0) return;
  std::vector<RegOp> rebuilt;
  for (int k = st0; k < st0 + nst; k++) {
    StageRec& st = out->stages[k];
    if (st.kind != 0) continue;
    const int op0 = first + (int)rebuilt.size();
    int i = st.op0;
    while (i < st.op0 + st.nops) {
      const RegOp& r = out->reg_ops[i];
      if (r.type != OP_RXT) {
        rebuilt.push_back(r);
        i++;
        continue;
      }
      uint32_t slots = 0;
      int e = i;
      while (e < st.op0 + st.nops && out->reg_ops[e].type == OP_RXT && !((slots >> out->reg_ops[e].s0) & 1u)) {
        slots |= 1u << out->reg_ops[e].s0;
        e++;
      }
      RegOp m;
      memset(&m, 0, sizeof(m));
      m.type = OP_RXTM;
      m.s0 = m.s1 = m.tb = -1;
      m.gbit = -1;
      m.csl = slots;
      m.mat = (int)out->pool.entries();
      for (int sl = 0; sl < 32; sl++)   // parameters in ascending slot order
        for (int q = i; q < e; q++)
          if (out->reg_ops[q].s0 == sl) {
            const RegOp& t = out->reg_ops[q];
            out->pool.add(cd(out->pool.f64[2 * (size_t)t.mat], 0.0));
            if (t.s1) m.neg |= (int8_t)(1 << sl);
          }
      rebuilt.push_back(m);
      i = e;
    }
    st.op0 = op0;
    st.nops = first + (int)rebuilt.size() - op0;
  }
  out->reg_ops.resize(first);
  out->reg_ops.insert(out->reg_ops.end(), rebuilt.begin(), rebuilt.end());
}

// The double-float tile kernels hold tile element i as (-i)^popcount(i) times its value
// (S^dagger on every tile bit; in that frame RX is a real rotation).  The general matrices
// of a pass move into the frame here: entry (r, c) of a gate on k tile bits (r, c indices
// over those bits) gets the factor (-i)^(popcount r - popcount c); controls cancel, rows
// and columns share them.  Full-form RX keeps its own kernel form, the real rotation
// [[c, s], [-s, c]], and gets c and s as two real entries; tangent-form RX, X (the kernel
// applies [[0, i], [-i, 0]]), SWAP and diagonal ops are unchanged.
namespace {

void times_mi_pow(Pool& pool, int entry, int e) {
  double& re = pool.f64[2 * (size_t)entry];
  double& im = pool.f64[2 * (size_t)entry + 1];
  const double a = re, b = im;
  switch (((e % 4) + 4) % 4) {
    case 1: re = b; im = -a; break;    // (-i)(a + ib) = b - ia
    case 2: re = -a; im = -b; break;
    case 3: re = -b; im = a; break;    // i(a + ib) = -b + ia
    default: break;
  }
}

void frame_block(Pool& pool, int mat, int k) {
  const int D = 1 << k;
  for (int r = 0; r < D; r++)
    for (int c = 0; c < D; c++) times_mi_pow(pool, mat + r * D + c, __builtin_popcount(r) - __builtin_popcount(c));
}

int split_rx(Pool& pool, int mat) {
  const double c = pool.f64[2 * (size_t)mat], sn = pool.f64[2 * (size_t)mat + 1];
  const int m = pool.add(cd(c, 0));
  pool.add(cd(sn, 0));
  return m;
}

}  // namespace

void apply_phase_frame(CompileResult* out, int st0, int nst) {
  for (int k = st0; k < st0 + nst; k++) {
    const StageRec& st = out->stages[k];
    for (int i = st.op0; i < st.op0 + st.nops; i++) {
      int32_t* mat;
      int type, nk = 0;
      if (st.kind == 1) {
        DevOp& o = out->tile_ops[i];
        mat = &o.mat;
        type = o.type;
        nk = o.nk;
      } else {
        RegOp& r = out->reg_ops[i];
        mat = &r.mat;
        type = r.type;
      }
      switch (type) {
        case OP_U1: frame_block(out->pool, *mat, 1); break;
        case OP_U2: frame_block(out->pool, *mat, 2); break;
        case OP_DENSE: frame_block(out->pool, *mat, nk); break;
        case OP_RX: *mat = split_rx(out->pool, *mat); break;
        default: break;
      }
    }
  }
}

int register_bits(int dtype, int L, int requested) {
  const int kmax = (dtype == QS_C128) ? 4 : 5;
  const int k = (requested > 0) ? std::min(requested, kmax) : kmax;
  return std::min(k, L);
}

// Working arrays of build_stages, kept per thread like merge_diagonals' (one call per pass).
struct StageScratch {
  std::vector<OpInfo> info;
  std::vector<std::vector<int>> preds;
  struct BS {
    int cls = -1;
    std::vector<int> cur, prev;
  };
  BS bs[32];
  std::vector<char> done, tmp;
  std::vector<uint32_t> okm;
  std::vector<int> rem, take;
  std::vector<RegOp> rl;
};

void build_stages(const std::vector<DevOp>& ops, int L, int K, CompileResult* out, int* st0, int* nst) {
  const int N = (int)ops.size();
  thread_local StageScratch ws;

  std::vector<OpInfo>& info = ws.info;
  info.resize(N);
  for (int i = 0; i < N; i++) {
    info[i] = classify_op(ops[i]);
    // an op whose non-diagonal bits outnumber the register bits (a 4x4 block with K = 1)
    // cannot run in registers
    if (__builtin_popcount(info[i].need) > K) info[i].smem_only = true;
  }
  // dependency DAG over tile bits (same grouping rule as the circuit DAG)
  std::vector<std::vector<int>>& preds = ws.preds;
  if (preds.size() < (size_t)N) preds.resize(N);
  for (int j = 0; j < N; j++) preds[j].clear();
  StageScratch::BS* bs = ws.bs;
  for (int b = 0; b < 32; b++) {
    bs[b].cls = -1;
    bs[b].cur.clear();
    bs[b].prev.clear();
  }
  for (int j = 0; j < N; j++) {
    for (int t = 0; t < info[j].nb; t++) {
      StageScratch::BS& s = bs[info[j].bit[t]];
      const int c = info[j].cls[t];
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
  std::vector<char>& done = ws.done;
  std::vector<char>& tmp = ws.tmp;
  done.assign(N, 0);
  tmp.assign(N, 0);
  std::vector<uint32_t>& okm = ws.okm;   // candidate-bit masks of the stage search
  okm.assign(N, 0);
  std::vector<int>& rem = ws.rem;
  rem.resize(N);
  for (int i = 0; i < N; i++) rem[i] = i;
  *st0 = (int)out->stages.size();
  auto ready = [&](int v) {
    for (int p : preds[v])
      if (!done[p]) return false;
    return true;
  };
  // ops one sweep schedules with register bits R (smem-only ops excluded)
  // a diagonal op on tile bits none of which is in R waits for a stage that holds one of
  // them, where it merges into the phase table; ops that depend on it act non-diagonally
  // on its bits and cannot run in this stage either
  int nondiag_left = 0;
  for (int v = 0; v < N; v++)
    if (info[v].need || info[v].smem_only) nondiag_left++;
  auto deferred = [&](int v, uint32_t R) {
    return !info[v].smem_only && info[v].need == 0 && info[v].tbits != 0 && (info[v].tbits & R) == 0 &&
           nondiag_left > 0;
  };
  // A stage's choice only looks at the first kWindow remaining ops: rem is in program order
  // and an op's predecessors come before it, so the count over that prefix is exact for the
  // ops in it, and the ops further on rarely change which register bits win.  It bounds the
  // search to O(kWindow) per candidate instead of O(ops in the pass).  256 and 768 give the
  // same plans on the 30-qubit construction and on 400 circuits of the batched workload.
  constexpr size_t kWindow = 256;
  while (!rem.empty()) {
    // the earliest ready op
    int first = -1;
    for (int v : rem)
      if (ready(v)) {
        first = v;
        break;
      }
    StageRec st;
    memset(&st, 0, sizeof(st));
    std::vector<int>& take = ws.take;
    take.clear();
    if (info[first].smem_only || K < 1) {
      st.kind = 1;
      // every ready shared-memory-only op (in program order, with intra-stage chaining)
      for (int v : rem) {
        if (!info[v].smem_only && K >= 1) continue;
        bool ok = true;
        for (int p : preds[v])
          if (!done[p] && !tmp[p]) {
            ok = false;
            break;
          }
        if (ok) {
          tmp[v] = 1;
          take.push_back(v);
        }
      }
      for (int v : take) tmp[v] = 0;
    } else {
      st.kind = 0;
      uint32_t R = 0;
      int nr = 0;
      // seed with the bits of the earliest ready op that needs registers
      for (int v : rem)
        if (!info[v].smem_only && info[v].need && ready(v)) {
          R = info[v].need;
          nr = __builtin_popcount(R);
          break;
        }
      while (nr < K) {
        // one sweep scores every candidate bit b at once: okm[v] has bit b set iff op v
        // would be scheduled with register bits R | b (its needs covered, not deferred,
        // every unfinished predecessor scheduled as well)
        const uint32_t all = (L >= 32) ? 0xFFFFFFFFu : ((1u << L) - 1u);
        const uint32_t cand = all & ~R;
        const size_t lim = std::min(rem.size(), kWindow);
        int score[32] = {0};
        int rank[32];
        for (int b = 0; b < 32; b++) rank[b] = 1 << 30;
        for (size_t r = 0; r < lim; r++) {
          const int v = rem[r];
          const OpInfo& in = info[v];
          uint32_t m = 0;
          if (!in.smem_only) {
            const uint32_t miss = in.need & ~R;
            m = (miss == 0) ? cand : ((miss & (miss - 1)) == 0 ? (miss & cand) : 0u);
            if (m && !in.need && in.tbits && nondiag_left > 0 && !(in.tbits & R)) m &= in.tbits;   // deferred unless b holds one of its bits
            for (int p : preds[v]) {
              if (!m) break;
              if (!done[p]) m &= okm[p];
            }
          }
          okm[v] = m;
          // an op that runs under every candidate adds the same to every score: skipped
          if (m != cand)
            for (uint32_t mm = m; mm; mm &= mm - 1) score[__builtin_ctz(mm)]++;
          for (uint32_t nb = in.need & cand; nb; nb &= nb - 1) {
            const int b = __builtin_ctz(nb);
            if (rank[b] == (1 << 30)) rank[b] = (int)r;
          }
        }
        int best = -1, best_s = -1, best_rank = 1 << 30;
        for (int b = 0; b < L; b++) {
          if ((R >> b) & 1u) continue;
          if (score[b] > best_s || (score[b] == best_s && rank[b] < best_rank)) {
            best = b;
            best_s = score[b];
            best_rank = rank[b];
          }
        }
        R |= 1u << best;
        nr++;
      }
      for (int v : rem) {
        bool ok = !info[v].smem_only && (info[v].need & ~R) == 0 && !deferred(v, R);
        if (ok)
          for (int p : preds[v])
            if (!done[p] && !tmp[p]) {
              ok = false;
              break;
            }
        if (ok) {
          tmp[v] = 1;
          take.push_back(v);
        }
      }
      for (int v : take) tmp[v] = 0;
      st.rmask = (int32_t)R;
      int k = 0;
      for (int b = 0; b < L; b++)
        if ((R >> b) & 1u) st.rbits[k++] = b;
    }
    // emit
    if (st.kind == 1) {
      st.op0 = (int)out->tile_ops.size();
      for (int v : take) out->tile_ops.push_back(ops[v]);
      st.nops = (int)take.size();
    } else {
      int slot[32];
      for (int b = 0; b < 32; b++) slot[b] = -1;
      for (int k = 0; k < K; k++) slot[st.rbits[k]] = k;
      const uint32_t R = (uint32_t)st.rmask;
      std::vector<RegOp>& rl = ws.rl;
      rl.clear();
      for (int v : take) {
        const DevOp& o = ops[v];
        RegOp r;
        memset(&r, 0, sizeof(r));
        r.type = o.type;
        r.s0 = r.s1 = r.tb = -1;
        r.gbit = -1;
        r.mat = o.mat;
        r.gmask = o.gmask;
        const uint32_t cm = (uint32_t)o.cmask;
        for (int b = 0; b < 32; b++)
          if ((cm >> b) & 1u) {
            if ((R >> b) & 1u) r.csl |= 1u << slot[b];
            else r.cot |= 1u << b;
          }
        switch (o.type) {
          case OP_U1: case OP_RX: case OP_X: r.s0 = (int8_t)slot[o.k0]; break;
          case OP_U2: r.s0 = (int8_t)slot[o.k0]; r.s1 = (int8_t)slot[o.k1]; break;
          case OP_DIAG:
            if (o.k0 >= 0) {
              if ((R >> o.k0) & 1u) r.s0 = (int8_t)slot[o.k0];
              else r.tb = (int8_t)o.k0;
            } else {
              r.gbit = o.gbit;
            }
            break;
          case OP_PHASE: r.neg = (o.mat < 0) ? 1 : 0; break;
          default: break;
        }
        if ((r.type == OP_U1 || r.type == OP_RX) && r.csl != 0) {
          // controlled 2x2 on a register slot: a 4x4 block on (target, control) slots,
          // index r = b(target) + 2 b(control), identity where the control is 0
          cd u[4];
          if (r.type == OP_U1) {
            for (int k = 0; k < 4; k++) u[k] = cd(out->pool.f64[2 * (r.mat + k)], out->pool.f64[2 * (r.mat + k) + 1]);
          } else {
            const double c = out->pool.f64[2 * r.mat], sn = out->pool.f64[2 * r.mat + 1];
            u[0] = c; u[1] = cd(0, -sn); u[2] = cd(0, -sn); u[3] = c;
          }
          int cs = 0;
          while (!((r.csl >> cs) & 1u)) cs++;
          r.type = OP_U2;
          r.s1 = (int8_t)cs;
          r.csl = 0;
          r.mat = (int)out->pool.entries();
          for (int a = 0; a < 4; a++)
            for (int b = 0; b < 4; b++) {
              cd v(0, 0);
              if (a < 2 && b < 2) v = (a == b) ? cd(1, 0) : cd(0, 0);
              else if (a >= 2 && b >= 2) v = u[(a - 2) * 2 + (b - 2)];
              out->pool.add(v);
            }
        }
        if (r.type == OP_U1 && r.csl == 0 && r.cot == 0 && r.gmask == 0) {
          // an uncontrolled general 2x2 in registers runs as diag . RX . diag: the diagonal
          // factors join the stage's phase tables and the RX takes the tangent form, about a
          // third of a general 2x2's arithmetic (shared-memory stages keep one op)
          cd u[4], d1[4], rx[4], d2[4];
          for (int k = 0; k < 4; k++) u[k] = cd(out->pool.f64[2 * (r.mat + k)], out->pool.f64[2 * (r.mat + k) + 1]);
          if (euler_split(u, d1, rx, d2)) {
            // the three factors take over the general matrix's four pool entries (its own):
            // the phase, the rotation (c, s), the two diagonal values
            auto put = [&](int k, const cd& z) {
              out->pool.f64[2 * (size_t)(r.mat + k)] = z.real();
              out->pool.f64[2 * (size_t)(r.mat + k) + 1] = z.imag();
            };
            RegOp p = r;
            if (d1[3] != cd(1, 0)) {   // diag(1, e^{i d}): a phase where the slot's bit is 1
              p.type = OP_PHASE;
              p.csl = 1u << r.s0;
              p.s0 = -1;
              p.neg = 0;
              put(0, d1[3]);
              rl.push_back(p);
            }
            p = r;
            p.type = OP_RX;
            p.mat = r.mat + 1;
            put(1, cd(rx[0].real(), -rx[1].imag()));
            rl.push_back(p);
            p = r;
            p.type = OP_DIAG;
            p.mat = r.mat + 2;
            put(2, d2[0]);
            put(3, d2[3]);
            rl.push_back(p);
            continue;
          }
        }
        rl.push_back(r);
      }
      merge_diagonals(rl, K, out->pool);
      st.op0 = (int)out->reg_ops.size();
      out->reg_ops.insert(out->reg_ops.end(), rl.begin(), rl.end());
      st.nops = (int)rl.size();
    }
    out->stages.push_back(st);
    for (int v : take) {
      done[v] = 1;
      if (info[v].need || info[v].smem_only) nondiag_left--;
    }
    size_t w = 0;
    for (size_t r = 0; r < rem.size(); r++)
      if (!done[rem[r]]) rem[w++] = rem[r];
    rem.resize(w);
  }
  *nst = (int)out->stages.size() - *st0;
  fold_pass_factors(out, *st0, *nst, K);
  merge_rxt_runs(out, *st0, *nst);
  if (out->pol == POL_DF) apply_phase_frame(out, *st0, *nst);
  // a thread keeps its arrays between passes, but not those of an unusually large one
  if (preds.size() > (1u << 16)) ws = StageScratch();
}

}  // namespace qs

namespace qs {

namespace {

// instructions per affected amplitude: {F32, F64 (DFMA), double-float}
struct Cost {
  double f32, f64, df;
};
double pick(const Cost& c, Policy p) { return p == POL_F32 ? c.f32 : (p == POL_F64 ? c.f64 : c.df); }

const Cost kRX{4, 4, 32};       // two real products and a sum per component
const Cost kRXT{2, 2, 24};      // one real product and a sum per component (tangent form)
const Cost kMUL{4, 4, 32};      // complex multiply (diagonal factor, table entry)
const Cost kU1{8, 8, 80};       // two complex products and a sum
const Cost kNEG{0, 0, 0};       // sign flips
// amplitude moves (X / CNOT targets, SWAP) do no arithmetic but cost instructions of the
// same order: register shuffles, and in the double-float phase frame a quarter-turn (lane
// swap and sign flips) of each moved amplitude.  Counted as instruction equivalents so that
// circuits made mostly of moves are not predicted free.
const Cost kMOVE{2, 2, 8};
const Cost kU2{16, 16, 172};    // per amplitude of a 4x4 block
const Cost kMACK{4, 4, 46};     // per amplitude per column of a 2^k block
const Cost kCONV{0, 0, 72};     // FP64 <-> (hi, lo) split / join per pass

double fraction(int bits) { return 1.0 / (double)(1u << bits); }

}  // namespace

double op_alu_per_amp(Policy pol, const DevOp& o) {
  const int ctl = __builtin_popcountll(o.cmask) + __builtin_popcountll(o.gmask);
  switch (o.type) {
    case OP_RX: return pick(kRX, pol) * fraction(ctl);
    case OP_U1: return pick(kU1, pol) * fraction(ctl);
    case OP_DIAG: return pick(kMUL, pol) * fraction(ctl);
    case OP_PHASE: return (o.mat < 0 ? pick(kNEG, pol) : pick(kMUL, pol)) * fraction(ctl);
    case OP_U2: return pick(kU2, pol) * fraction(ctl);
    case OP_DENSE: return pick(kMACK, pol) * (double)(1 << o.nk) * fraction(ctl);
    case OP_X: return pick(kMOVE, pol) * fraction(ctl);
    case OP_SWAP: return pick(kMOVE, pol) * fraction(ctl + 1);
    default: return 0.0;
  }
}

double stage_alu_per_amp(const CompileResult& cr, int st0, int nst) {
  double a = pick(kCONV, cr.pol);
  for (int k = st0; k < st0 + nst; k++) {
    const StageRec& st = cr.stages[k];
    if (st.kind == 1) {
      for (int i = st.op0; i < st.op0 + st.nops; i++) a += op_alu_per_amp(cr.pol, cr.tile_ops[i]);
      continue;
    }
    for (int i = st.op0; i < st.op0 + st.nops; i++) {
      const RegOp& r = cr.reg_ops[i];
      const int ctl = __builtin_popcount(r.csl) + __builtin_popcount(r.cot) + __builtin_popcountll(r.gmask);
      switch (r.type) {
        case OP_RX: a += pick(kRX, cr.pol) * fraction(ctl); break;
        case OP_RXT: a += pick(kRXT, cr.pol) * fraction(ctl); break;
        case OP_RXTM: a += pick(kRXT, cr.pol) * (double)__builtin_popcount(r.csl); break;
        case OP_U1: a += pick(kU1, cr.pol) * fraction(ctl); break;
        case OP_DIAG: a += pick(kMUL, cr.pol) * fraction(ctl); break;
        case OP_DTAB:   // double-float / FP64 multiply only the entries that are not exactly 1
          a += pick(kMUL, cr.pol) * (cr.pol == POL_F32 ? 1.0
                                                        : (double)__builtin_popcount(r.csl) /
                                                              (double)(1u << __builtin_popcount((uint32_t)st.rmask)));
          break;
        case OP_PHASE: a += (r.neg ? pick(kNEG, cr.pol) : pick(kMUL, cr.pol)) * fraction(ctl); break;
        case OP_U2: a += pick(kU2, cr.pol) * fraction(ctl); break;
        case OP_X: a += pick(kMOVE, cr.pol) * fraction(ctl); break;
        default: break;
      }
    }
  }
  return a;
}

double gate_tile_alu_per_amp(Policy pol, const HGate& g) {
  bool diag = true;
  for (int t = 0; t < g.nq; t++) diag &= g.cls[t] == CLS_Z;
  int ctl = 0;   // controls restrict the amplitudes touched
  if (g.kind == QS_OP_CNOT || g.kind == QS_OP_CU || g.kind == QS_OP_CP) ctl = 1;
  if (diag) {
    if (g.kind == QS_OP_CZ || g.kind == QS_OP_Z) return 0.0;   // sign flips
    // diagonal factors merge into register phase tables, typically two or more per table
    return 0.5 * pick(kMUL, pol) * fraction(g.nq >= 2 ? g.nq - 1 : 0);
  }
  if (g.nq == 1) {   // by form: fused products are U1 gates whatever their matrix
    const cd* m = g.U.data();
    if (m[0] == cd(0, 0) && m[3] == cd(0, 0) && m[1] == cd(1, 0) && m[2] == cd(1, 0)) return pick(kMOVE, pol);
    if (m[0] == m[3] && m[0].imag() == 0.0 && m[1] == m[2] && m[1].real() == 0.0) return pick(kRXT, pol);
    // a general 2x2 runs in registers as diag . RX . diag, its two factors in phase tables
    return pick(kRXT, pol) + pick(kMUL, pol);
  }
  if (g.kind == QS_OP_CNOT) return pick(kMOVE, pol) * fraction(1);
  if (g.kind == QS_OP_SWAP) return pick(kMOVE, pol) * fraction(1);
  if (g.kind == QS_OP_CU) return pick(kU1, pol) * fraction(ctl);
  if (g.nq == 2) return pick(kU2, pol);
  return pick(kMACK, pol) * (double)(1 << g.nq);
}

}  // namespace qs
