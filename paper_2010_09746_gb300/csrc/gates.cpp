// Host gate model: ABI op -> matrix + per-qubit action classes, lowering to device ops,
// and the policy-specific serialisation of matrix pools.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "qs_internal.h"

namespace qs {

namespace {

const double kInvSqrt2 = 0.70710678118654752440;

bool one_qubit(int kind, double t, cd m[4]) {
  const cd I(0, 1);
  switch (kind) {
    case QS_OP_H: m[0] = kInvSqrt2; m[1] = kInvSqrt2; m[2] = kInvSqrt2; m[3] = -kInvSqrt2; return true;
    case QS_OP_X: m[0] = 0; m[1] = 1; m[2] = 1; m[3] = 0; return true;
    case QS_OP_Y: m[0] = 0; m[1] = -I; m[2] = I; m[3] = 0; return true;
    case QS_OP_Z: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = -1; return true;
    case QS_OP_S: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = I; return true;
    case QS_OP_T: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = cd(kInvSqrt2, kInvSqrt2); return true;
    case QS_OP_RZ: m[0] = cd(cos(0.5 * t), -sin(0.5 * t)); m[1] = 0; m[2] = 0; m[3] = cd(cos(0.5 * t), sin(0.5 * t)); return true;
    case QS_OP_RX: m[0] = cos(0.5 * t); m[1] = cd(0, -sin(0.5 * t)); m[2] = cd(0, -sin(0.5 * t)); m[3] = cos(0.5 * t); return true;
    case QS_OP_RY: m[0] = cos(0.5 * t); m[1] = -sin(0.5 * t); m[2] = sin(0.5 * t); m[3] = cos(0.5 * t); return true;
    case QS_OP_P: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = cd(cos(t), sin(t)); return true;
    default: return false;
  }
}

// classes by exact commutation with Z / X on each qubit of a 2^k x 2^k matrix
void classify(HGate* g) {
  const int D = 1 << g->nq;
  for (int t = 0; t < g->nq; t++) {
    const int bq = 1 << t;
    bool diag = true, xtype = true;
    for (int r = 0; r < D && (diag || xtype); r++)
      for (int c = 0; c < D; c++) {
        const cd u = g->U[(size_t)r * D + c];
        if (((r ^ c) & bq) && u != cd(0, 0)) diag = false;
        if (u != g->U[(size_t)(r ^ bq) * D + (c ^ bq)]) xtype = false;
      }
    g->cls[t] = diag ? CLS_Z : (xtype ? CLS_X : CLS_N);
  }
}

}  // namespace

bool make_hgate(int n, const qs_op& op, const double* mats, size_t nmats, HGate* g, std::string* err) {
  g->kind = op.kind;
  g->param = op.param;
  int nq;
  switch (op.kind) {
    case QS_OP_U1: case QS_OP_H: case QS_OP_X: case QS_OP_Y: case QS_OP_Z: case QS_OP_S: case QS_OP_T:
    case QS_OP_RZ: case QS_OP_RX: case QS_OP_RY: case QS_OP_P:
      nq = 1; break;
    case QS_OP_CNOT: case QS_OP_CZ: case QS_OP_CP: case QS_OP_CU: case QS_OP_SWAP: case QS_OP_U2:
    case QS_OP_RELABEL:
      nq = 2; break;
    case QS_OP_UK:
      nq = op.nq;
      if (nq < 1 || nq > kMaxDenseK) { *err = "UK gate needs 1 <= nq <= 6"; return false; }
      break;
    default:
      *err = "unknown gate kind " + std::to_string(op.kind);
      return false;
  }
  if (op.nq != nq) { *err = "gate kind " + std::to_string(op.kind) + " needs nq = " + std::to_string(nq); return false; }
  g->nq = nq;
  for (int t = 0; t < nq; t++) {
    if (op.q[t] < 0 || op.q[t] >= n) { *err = "qubit index out of range"; return false; }
    for (int s = 0; s < t; s++)
      if (op.q[s] == op.q[t]) { *err = "duplicate qubit in gate"; return false; }
    g->q[t] = op.q[t];
  }
  const int D = 1 << nq;
  g->U.assign((size_t)D * D, cd(0, 0));
  auto need_mat = [&](size_t count) -> const double* {
    if (op.mat < 0 || mats == nullptr || (size_t)op.mat + count > nmats) return nullptr;
    return mats + op.mat;
  };
  cd m[4];
  if (nq == 1 && op.kind != QS_OP_UK) {
    if (op.kind == QS_OP_U1) {
      const double* p = need_mat(8);
      if (!p) { *err = "U1 gate matrix offset out of range"; return false; }
      for (int k = 0; k < 4; k++) m[k] = cd(p[2 * k], p[2 * k + 1]);
    } else {
      one_qubit(op.kind, op.param, m);
    }
    for (int k = 0; k < 4; k++) g->U[k] = m[k];
  } else if (op.kind == QS_OP_CNOT || op.kind == QS_OP_CZ || op.kind == QS_OP_CP || op.kind == QS_OP_CU) {
    if (op.kind == QS_OP_CU) {
      const double* p = need_mat(8);
      if (!p) { *err = "CU gate matrix offset out of range"; return false; }
      for (int k = 0; k < 4; k++) m[k] = cd(p[2 * k], p[2 * k + 1]);
    } else {
      one_qubit(op.kind == QS_OP_CNOT ? QS_OP_X : (op.kind == QS_OP_CZ ? QS_OP_Z : QS_OP_P), op.param, m);
    }
    // r = b(control) + 2 b(target); control = 1 rows/cols are 1 and 3
    g->U[0 * 4 + 0] = 1;
    g->U[2 * 4 + 2] = 1;
    g->U[1 * 4 + 1] = m[0];
    g->U[1 * 4 + 3] = m[1];
    g->U[3 * 4 + 1] = m[2];
    g->U[3 * 4 + 3] = m[3];
  } else if (op.kind == QS_OP_SWAP || op.kind == QS_OP_RELABEL) {
    g->U[0] = 1; g->U[1 * 4 + 2] = 1; g->U[2 * 4 + 1] = 1; g->U[15] = 1;
  } else {   // U2, UK
    const double* p = need_mat((size_t)2 * D * D);
    if (!p) { *err = "gate matrix offset out of range"; return false; }
    for (int k = 0; k < D * D; k++) g->U[k] = cd(p[2 * k], p[2 * k + 1]);
  }
  classify(g);
  return true;
}

HGate make_1q_gate(int q, const cd m[4]) {
  HGate g;
  g.kind = QS_OP_U1;
  g.nq = 1;
  g.q[0] = q;
  g.param = 0.0;
  g.U.assign(m, m + 4);
  classify(&g);
  return g;
}

size_t Pool::entry_bytes(Policy pol) { return pol == POL_F32 ? 8 : (pol == POL_F64 ? 16 : 48); }

void Pool::serialise_into(Policy pol, unsigned char* dst) const {
  const size_t E = entries();
  if (pol == POL_F32) {
    float* f = (float*)dst;
    for (size_t k = 0; k < E; k++) {
      f[2 * k] = (float)f64[2 * k];
      f[2 * k + 1] = (float)f64[2 * k + 1];
    }
  } else if (pol == POL_F64) {
    memcpy(dst, f64.data(), E * 16);
  } else {
    // double-float lane patterns of u = ur + i ui (12 floats): (ur, ur) and its negation,
    // (-ui, ui) and its negation, then the negated low parts of (ur, ur) and (-ui, ui)
    float* f = (float*)dst;
    for (size_t k = 0; k < E; k++) {
      const double ur = f64[2 * k], ui = f64[2 * k + 1];
      const float rh = (float)ur, rl = (float)(ur - (double)rh);
      const float ih = (float)ui, il = (float)(ui - (double)ih);
      float* e = f + 12 * k;
      e[0] = rh; e[1] = rh; e[2] = -rh; e[3] = -rh;
      e[4] = -ih; e[5] = ih; e[6] = ih; e[7] = -ih;
      e[8] = -rl; e[9] = -rl; e[10] = il; e[11] = -il;
    }
  }
}

std::vector<unsigned char> Pool::serialise(Policy pol) const {
  std::vector<unsigned char> out(entries() * entry_bytes(pol));
  if (!out.empty()) serialise_into(pol, out.data());
  return out;
}

// ------------------------------------------------------------------------------------------
// Lowering
// ------------------------------------------------------------------------------------------
namespace {

struct Addr {
  bool ok;
  int idx;          // bit index in the addressed space (tile-local or storage), -1 if outside
  int storage;      // storage bit
};

Addr addr_of(const LowerCtx& ctx, int q) {
  Addr a;
  a.storage = ctx.sigma[q];
  if (ctx.tile) {
    a.idx = ctx.tile_index[a.storage];
    a.ok = a.idx >= 0;
  } else {
    a.idx = a.storage;
    a.ok = true;
  }
  return a;
}

DevOp blank() {
  DevOp o;
  memset(&o, 0, sizeof(o));
  o.k0 = o.k1 = -1;
  o.mat = -1;
  o.gbit = -1;
  return o;
}

// add a control on logical qubit q (addressable -> cmask, else gmask)
void add_ctrl(const LowerCtx& ctx, int q, DevOp* o) {
  Addr a = addr_of(ctx, q);
  if (a.ok) o->cmask |= 1ull << a.idx;
  else o->gmask |= 1ull << a.storage;
}

bool is_real(const cd& z) { return z.imag() == 0.0; }

// out = a b for row-major 2x2 matrices
void mul2x2(const cd a[4], const cd b[4], cd out[4]) {
  const cd r0 = a[0] * b[0] + a[1] * b[2], r1 = a[0] * b[1] + a[1] * b[3];
  const cd r2 = a[2] * b[0] + a[3] * b[2], r3 = a[2] * b[1] + a[3] * b[3];
  out[0] = r0;
  out[1] = r1;
  out[2] = r2;
  out[3] = r3;
}

// Euler form of a U(2) matrix about the Z and X axes: U = e^{i a} RZ(b) RX(t) RZ(d) for every
// unitary U.  Written as U = D2 RX(t) D1 with D1 = diag(1, e^{i d}) (RZ(d) up to the scalar
// e^{-i d / 2}) and D2 = e^{i (a - d / 2)} RZ(b), so that the RX factor has the exact
// structure c I - i s X (OP_RX).  With e^{i a} = sqrt(det U) and
// V = e^{-i a} U = [[v, w], [-w*, v*]] in SU(2): v = cos(t/2) A and w = -i sin(t/2) B with
// the unit numbers A = e^{-i (b + d)/2}, B = e^{-i (b - d)/2}; so e^{i d} = A* B and
// D2 = e^{i a} diag(A, B*), all from complex arithmetic without angles.  False when the
// three factors miss U by more than 1e-13 in some entry (U not unitary enough); the
// caller then applies U as one general matrix.
bool euler_zxz(const cd U[4], cd d1[4], cd rx[4], cd d2[4]) {
  const cd ea = std::sqrt(U[0] * U[3] - U[1] * U[2]);
  if (!(std::abs(ea) > 0)) return false;
  const cd v00 = U[0] / ea, v01 = U[1] / ea;
  const double av = std::abs(v00), aw = std::abs(v01), r = std::hypot(av, aw);
  if (!(r > 0)) return false;
  const double c = av / r, s = aw / r;
  const cd A = av > 0 ? v00 / av : cd(1, 0);
  const cd B = aw > 0 ? cd(0, 1) * v01 / aw : cd(1, 0);
  d1[0] = 1; d1[1] = 0; d1[2] = 0; d1[3] = std::conj(A) * B;
  rx[0] = c; rx[1] = cd(0, -s); rx[2] = cd(0, -s); rx[3] = c;
  d2[0] = ea * A; d2[1] = 0; d2[2] = 0; d2[3] = ea * std::conj(B);
  cd t[4], w[4];
  mul2x2(rx, d1, t);
  mul2x2(d2, t, w);
  for (int k = 0; k < 4; k++)
    if (std::abs(w[k] - U[k]) > 1e-13) return false;
  return true;
}

// 2x2 matrix m on logical qubit t with controls ctrls
bool lower_2x2(const cd m[4], int t, const int* ctrls, int nc, const LowerCtx& ctx, Pool& pool,
               std::vector<DevOp>& out) {
  DevOp o = blank();
  for (int k = 0; k < nc; k++) add_ctrl(ctx, ctrls[k], &o);
  Addr a = addr_of(ctx, t);
  const bool diag = m[1] == cd(0, 0) && m[2] == cd(0, 0);
  if (diag) {
    if (m[0] == cd(1, 0)) {
      if (m[3] == cd(1, 0)) return true;   // identity
      // phase on bit t = 1
      if (a.ok) o.cmask |= 1ull << a.idx;
      else o.gmask |= 1ull << a.storage;
      o.type = OP_PHASE;
      o.mat = (m[3] == cd(-1, 0)) ? -1 : pool.add(m[3]);
      out.push_back(o);
      return true;
    }
    o.type = OP_DIAG;
    o.mat = pool.add(m[0]);
    pool.add(m[3]);
    if (a.ok) {
      o.k0 = a.idx;
    } else {
      if (!ctx.tile) return false;
      o.k0 = -1;
      o.gbit = a.storage;
    }
    out.push_back(o);
    return true;
  }
  if (!a.ok) return false;   // non-diagonal target must be addressable
  o.k0 = a.idx;
  if (m[0] == cd(0, 0) && m[3] == cd(0, 0) && m[1] == cd(1, 0) && m[2] == cd(1, 0)) {
    o.type = OP_X;
    out.push_back(o);
    return true;
  }
  if (m[0] == m[3] && is_real(m[0]) && m[1] == m[2] && m[1].real() == 0.0) {
    o.type = OP_RX;   // c I - i s X
    o.mat = pool.add(cd(m[0].real(), -m[1].imag()));
    out.push_back(o);
    return true;
  }
  o.type = OP_U1;
  o.mat = pool.add(m[0]);
  pool.add(m[1]);
  pool.add(m[2]);
  pool.add(m[3]);
  out.push_back(o);
  return true;
}

}  // namespace

bool euler_split(const cd U[4], cd d1[4], cd rx[4], cd d2[4]) { return euler_zxz(U, d1, rx, d2); }

bool lower_gate(const HGate& g, const LowerCtx& ctx, Pool& pool, std::vector<DevOp>& out) {
  const int D = 1 << g.nq;
  if (g.nq == 1) {
    cd m[4] = {g.U[0], g.U[1], g.U[2], g.U[3]};
    return lower_2x2(m, g.q[0], nullptr, 0, ctx, pool, out);
  }
  if (g.kind == QS_OP_CNOT || g.kind == QS_OP_CZ || g.kind == QS_OP_CP || g.kind == QS_OP_CU) {
    cd m[4] = {g.U[1 * 4 + 1], g.U[1 * 4 + 3], g.U[3 * 4 + 1], g.U[3 * 4 + 3]};
    int c = g.q[0];
    return lower_2x2(m, g.q[1], &c, 1, ctx, pool, out);
  }
  if (g.kind == QS_OP_SWAP) {
    Addr a = addr_of(ctx, g.q[0]), b = addr_of(ctx, g.q[1]);
    if (!a.ok || !b.ok) return false;
    DevOp o = blank();
    o.type = OP_SWAP;
    o.k0 = std::min(a.idx, b.idx);
    o.k1 = std::max(a.idx, b.idx);
    out.push_back(o);
    return true;
  }
  // general 2-qubit / k-qubit dense: every qubit must be addressable
  DevOp o = blank();
  int idx[kMaxDenseK];
  for (int t = 0; t < g.nq; t++) {
    Addr a = addr_of(ctx, g.q[t]);
    if (!a.ok) return false;
    idx[t] = a.idx;
  }
  o.mat = (int)pool.entries();
  for (int k = 0; k < D * D; k++) pool.add(g.U[k]);
  if (g.nq == 2) {
    o.type = OP_U2;
    o.k0 = idx[0];
    o.k1 = idx[1];
  } else {
    o.type = OP_DENSE;
    o.nk = g.nq;
    for (int t = 0; t < g.nq; t++) o.kq[t] = idx[t];
  }
  out.push_back(o);
  return true;
}

// The real 128 x 128 matrix of a dense k-qubit block on storage bits bits[0..k-1] (a
// permutation of 0..k-1), replicated over storage bits k..5, transposed (row j = output
// float j of a 64-amplitude row) and split into its nearest TF32 values and the TF32-rounded
// remainders.
void dense_mma_weights(const double* U, int k, const int* bits, float* out) {
  const int kdim = 1 << k;
  const int mask = kdim - 1;
  auto mat_index = [&](int x) {
    int r = 0;
    for (int t = 0; t < k; t++) r |= ((x >> bits[t]) & 1) << t;
    return r;
  };
  std::vector<double> wt(128 * 128, 0.0);
  for (int xr = 0; xr < 64; xr++)
    for (int xc = 0; xc < 64; xc++) {
      if ((xr & ~mask) != (xc & ~mask)) continue;
      const int r = mat_index(xr & mask), c = mat_index(xc & mask);
      const double a = U[2 * (r * kdim + c)], b = U[2 * (r * kdim + c) + 1];
      wt[(2 * xr) * 128 + 2 * xc] = a;
      wt[(2 * xr) * 128 + 2 * xc + 1] = -b;
      wt[(2 * xr + 1) * 128 + 2 * xc] = b;
      wt[(2 * xr + 1) * 128 + 2 * xc + 1] = a;
    }
  auto tf32_rna = [](double v) {   // nearest TF32 value (ties away from zero), as a float
    const float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
  };
  for (int i = 0; i < 128 * 128; i++) {
    const float big = tf32_rna(wt[i]);
    out[i] = big;
    out[128 * 128 + i] = tf32_rna(wt[i] - (double)big);
  }
}


}  // namespace qs
