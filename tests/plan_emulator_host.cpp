// Host emulation of compiled plans, for the CPU tests of the compiler.
//
// It compiles a circuit with the library's own host compiler (make_hgate, compile_circuit:
// DAG, Algorithm 1, tile scheduler, register stages, phase tables, tangent-form RX, the
// double-float phase frame). It then executes the resulting steps in std::complex<double>
// with the kernels' documented op semantics. The test compares the final state with the
// FP64 oracle: a scheduling, lowering, folding or frame error shows up as an O(1)
// difference, far above the emulation's rounding. It is test infrastructure: the product
// path runs only on the GPU kernels.
//
// Input (binary file, argv[1]): int32 n, int32 nops, int64 nmats, qs_compile_opts, nops
// qs_op records, nmats doubles. Output (binary file, argv[2]): int32 n, int32 nsteps,
// int32 sigma_final[n], then 2^n complex doubles in storage order.
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../paper_2010_09746_gb300/csrc/qs_internal.h"

namespace qs {
void set_last_error(const std::string&) {}
}  // namespace qs

using namespace qs;
typedef std::complex<double> C;

static C entry(const Pool& p, int k) { return C(p.f64[2 * (size_t)k], p.f64[2 * (size_t)k + 1]); }
static C mi_pow(int q) {   // (-i)^q
  switch (q & 3) {
    case 0: return C(1, 0);
    case 1: return C(0, -1);
    case 2: return C(-1, 0);
    default: return C(0, 1);
  }
}
static int popc(uint64_t v) { return __builtin_popcountll(v); }
static uint64_t bit(uint64_t v, int b) { return (v >> b) & 1ull; }

// Shared-memory tile op or per-gate op on the index bits of T (tile-local or storage bits).
// `frame`: the double-float tile pass's S-dagger phase frame (RX real rotation with entries
// (c, 0), (s, 0); X as [[0, i], [-i, 0]]).
static void dev_op(std::vector<C>& T, const DevOp& op, const Pool& pool, uint64_t base, bool tile, bool frame) {
  if (tile && (base & op.gmask) != op.gmask) return;
  const uint64_t N = T.size(), cm = op.cmask;
  auto ctl = [&](uint64_t i) { return (i & cm) == cm; };
  switch (op.type) {
    case OP_U1:
    case OP_RX: {
      const uint64_t s = 1ull << op.k0;
      for (uint64_t i = 0; i < N; i++) {
        if ((i & s) || !ctl(i)) continue;
        const C a = T[i], b = T[i | s];
        if (op.type == OP_U1) {
          T[i] = entry(pool, op.mat) * a + entry(pool, op.mat + 1) * b;
          T[i | s] = entry(pool, op.mat + 2) * a + entry(pool, op.mat + 3) * b;
        } else if (frame) {
          const double c = entry(pool, op.mat).real(), sn = entry(pool, op.mat + 1).real();
          T[i] = c * a + sn * b;
          T[i | s] = c * b - sn * a;
        } else {
          const double c = entry(pool, op.mat).real(), sn = entry(pool, op.mat).imag();
          T[i] = c * a - C(0, sn) * b;
          T[i | s] = c * b - C(0, sn) * a;
        }
      }
      break;
    }
    case OP_DIAG: {
      const C d0 = entry(pool, op.mat), d1 = entry(pool, op.mat + 1);
      for (uint64_t i = 0; i < N; i++) {
        if (!ctl(i)) continue;
        const bool one = op.k0 >= 0 ? bit(i, op.k0) : bit(base, op.gbit);
        T[i] *= one ? d1 : d0;
      }
      break;
    }
    case OP_PHASE:
      for (uint64_t i = 0; i < N; i++) {
        if (!ctl(i)) continue;
        T[i] = op.mat < 0 ? -T[i] : T[i] * entry(pool, op.mat);
      }
      break;
    case OP_X:
    case OP_SWAP: {
      const uint64_t s0 = op.type == OP_X ? 0 : 1ull << op.k0;
      const uint64_t s1 = op.type == OP_X ? 1ull << op.k0 : 1ull << op.k1;
      for (uint64_t i = 0; i < N; i++) {
        if ((i & (s0 | s1)) || !ctl(i)) continue;
        const C a = T[i | s0], b = T[i | s1];
        const bool fx = frame && op.type == OP_X;
        T[i | s0] = fx ? C(0, 1) * b : b;
        T[i | s1] = fx ? C(0, -1) * a : a;
      }
      break;
    }
    case OP_U2:
    case OP_DENSE: {
      int k = 2, q[8] = {op.k0, op.k1};
      if (op.type == OP_DENSE) {
        k = op.nk;
        for (int t = 0; t < k; t++) q[t] = op.kq[t];
      }
      const int D = 1 << k;
      uint64_t zb = 0;
      for (int t = 0; t < k; t++) zb |= 1ull << q[t];
      std::vector<C> x(D), y(D);
      std::vector<uint64_t> off(D);
      for (int r = 0; r < D; r++) {
        off[r] = 0;
        for (int t = 0; t < k; t++)
          if ((r >> t) & 1) off[r] |= 1ull << q[t];
      }
      for (uint64_t i = 0; i < N; i++) {
        if ((i & zb) || !ctl(i)) continue;
        for (int r = 0; r < D; r++) x[r] = T[i | off[r]];
        for (int r = 0; r < D; r++) {
          y[r] = 0;
          for (int c = 0; c < D; c++) y[r] += entry(pool, op.mat + r * D + c) * x[c];
        }
        for (int r = 0; r < D; r++) T[i | off[r]] = y[r];
      }
      break;
    }
    default:
      fprintf(stderr, "unknown device op %d\n", op.type);
      exit(3);
  }
}

// Tangent-form RX on register slot S: mode 0 is cos-factored, mode 1 sin-factored.
static void reg_rxt(std::vector<C>& x, int S, double t, int mode, bool frame) {
  const int s = 1 << S;
  for (int j = 0; j < (int)x.size(); j++) {
    if (j & s) continue;
    const C a = x[j], b = x[j | s];
    if (frame) {   // [[1, t], [-t, 1]] or [[t, 1], [-1, t]]
      x[j] = mode == 0 ? a + t * b : t * a + b;
      x[j | s] = mode == 0 ? b - t * a : t * b - a;
    } else {       // I - i t X or t I - i X
      const C mi(0, -1);
      x[j] = mode == 0 ? a + t * mi * b : t * a + mi * b;
      x[j | s] = mode == 0 ? b + t * mi * a : t * b + mi * a;
    }
  }
}

static void reg_op(std::vector<C>& x, const RegOp& op, const Pool& pool, uint32_t gidx, uint64_t base, bool frame) {
  if ((gidx & op.cot) != op.cot) return;
  const int D = (int)x.size();
  const uint32_t csl = op.csl;
  auto ctl = [&](int j) { return ((uint32_t)j & csl) == csl; };
  switch (op.type) {
    case OP_U1: {
      const int s = 1 << op.s0;
      for (int j = 0; j < D; j++) {
        if (j & s) continue;
        const C a = x[j], b = x[j | s];
        x[j] = entry(pool, op.mat) * a + entry(pool, op.mat + 1) * b;
        x[j | s] = entry(pool, op.mat + 2) * a + entry(pool, op.mat + 3) * b;
      }
      break;
    }
    case OP_RX: {
      const int s = 1 << op.s0;
      for (int j = 0; j < D; j++) {
        if (j & s) continue;
        const C a = x[j], b = x[j | s];
        if (frame) {
          const double c = entry(pool, op.mat).real(), sn = entry(pool, op.mat + 1).real();
          x[j] = c * a + sn * b;
          x[j | s] = c * b - sn * a;
        } else {
          const double c = entry(pool, op.mat).real(), sn = entry(pool, op.mat).imag();
          x[j] = c * a - C(0, sn) * b;
          x[j | s] = c * b - C(0, sn) * a;
        }
      }
      break;
    }
    case OP_RXT:
      reg_rxt(x, op.s0, entry(pool, op.mat).real(), op.s1, frame);
      break;
    case OP_RXTM: {
      int idx = 0;
      for (int sl = 0; sl < 32; sl++)
        if ((csl >> sl) & 1u) {
          reg_rxt(x, sl, entry(pool, op.mat + idx).real(), ((uint8_t)op.neg >> sl) & 1, frame);
          idx++;
        }
      break;
    }
    case OP_X: {
      const int s = 1 << op.s0;
      for (int j = 0; j < D; j++) {
        if ((j & s) || !ctl(j)) continue;
        const C a = x[j], b = x[j | s];
        x[j] = frame ? C(0, 1) * b : b;
        x[j | s] = frame ? C(0, -1) * a : a;
      }
      break;
    }
    case OP_U2: {
      const int s0 = 1 << op.s0, s1 = 1 << op.s1;
      for (int j = 0; j < D; j++) {
        if ((j & (s0 | s1)) || (csl && !ctl(j))) continue;
        const int idx[4] = {j, j | s0, j | s1, j | s0 | s1};
        C v[4], y[4];
        for (int r = 0; r < 4; r++) v[r] = x[idx[r]];
        for (int r = 0; r < 4; r++) {
          y[r] = 0;
          for (int c = 0; c < 4; c++) y[r] += entry(pool, op.mat + 4 * r + c) * v[c];
        }
        for (int r = 0; r < 4; r++) x[idx[r]] = y[r];
      }
      break;
    }
    case OP_DIAG: {
      const C d0 = entry(pool, op.mat), d1 = entry(pool, op.mat + 1);
      for (int j = 0; j < D; j++) {
        if (!ctl(j)) continue;
        bool one;
        if (op.s0 >= 0) one = (j >> op.s0) & 1;
        else if (op.tb >= 0) one = (gidx >> op.tb) & 1u;
        else one = bit(base, op.gbit);
        x[j] *= one ? d1 : d0;
      }
      break;
    }
    case OP_DTAB:
      for (int j = 0; j < D; j++)
        if ((csl >> j) & 1u) x[j] *= entry(pool, op.mat + j);
      break;
    case OP_PHASE:
      for (int j = 0; j < D; j++) {
        if (!ctl(j)) continue;
        x[j] = op.neg ? -x[j] : x[j] * entry(pool, op.mat);
      }
      break;
    default:
      fprintf(stderr, "unknown register op %d\n", op.type);
      exit(3);
  }
}

// largest |amplitude| held in registers after any register op (scaled tangent-form updates
// let it grow above 1 inside a pass; the kernels need it to stay well inside FP32 range)
static double g_max_abs = 0;

static void run_pass(std::vector<C>& psi, const CompileResult& cr, const TilePass& tp) {
  const int L = tp.L, n = tp.n;
  const bool frame = cr.pol == POL_DF;
  const uint64_t nt = 1ull << L, nblocks = 1ull << (n - L);
  std::vector<C> T(nt);
  std::vector<uint64_t> addr(nt);
  std::vector<C> out(psi.size());
  for (uint64_t b = 0; b < nblocks; b++) {
    uint64_t base = 0;
    for (int k = 0; k < n - L; k++)
      if (bit(b, k)) base |= 1ull << tp.npos[k];
    for (uint64_t i = 0; i < nt; i++) {
      uint64_t a = base;
      for (int k = 0; k < L; k++)
        if (bit(i, k)) a |= 1ull << tp.tpos[k];
      addr[i] = a;
      T[i] = psi[a] * (frame ? mi_pow(popc(i)) : C(1, 0));
    }
    for (int s = tp.st0; s < tp.st0 + tp.nst; s++) {
      const StageRec& st = cr.stages[s];
      if (st.kind == 1) {
        for (int o = st.op0; o < st.op0 + st.nops; o++) dev_op(T, cr.tile_ops[o], cr.pool, base, true, frame);
        continue;
      }
      const uint32_t rmask = (uint32_t)st.rmask;
      const int K = __builtin_popcount(rmask);   // rbits[0..K) lists those bits in slot order
      std::vector<C> x(1u << K);
      for (uint64_t g = 0; g < nt; g++) {
        if (g & rmask) continue;
        const uint32_t gidx = (uint32_t)g;
        for (int j = 0; j < (1 << K); j++) {
          uint64_t i = gidx;
          for (int t = 0; t < K; t++)
            if ((j >> t) & 1) i |= 1ull << st.rbits[t];
          x[j] = T[i];
        }
        for (int o = st.op0; o < st.op0 + st.nops; o++) {
          const RegOp& op = cr.reg_ops[o];
          if ((base & op.gmask) != op.gmask) continue;
          reg_op(x, op, cr.pool, gidx, base, frame);
          for (const C& v : x) g_max_abs = std::max(g_max_abs, std::abs(v));
        }
        for (int j = 0; j < (1 << K); j++) {
          uint64_t i = gidx;
          for (int t = 0; t < K; t++)
            if ((j >> t) & 1) i |= 1ull << st.rbits[t];
          T[i] = x[j];
        }
      }
    }
    // the store, with the exchange of storage bits swap_a / swap_b of a fused PermuteQubits
    // (into a separate output vector, as the kernel writes to the other buffer)
    for (uint64_t i = 0; i < nt; i++) {
      uint64_t a = addr[i];
      const uint64_t d = ((a >> tp.swap_a) ^ (a >> tp.swap_b)) & 1ull;
      a ^= (d << tp.swap_a) | (d << tp.swap_b);
      out[a] = T[i] * (frame ? mi_pow(-popc(i)) : C(1, 0));
    }
  }
  psi.swap(out);
}

// `--euler in.bin out.bin`: the library's Euler split of each 2x2 matrix in in.bin (count,
// then 8 doubles per matrix, row-major re/im), written as a status and the three factors
// (d1, rx, d2; 8 doubles each) per matrix, for the test to check against numpy.
// Every field of a compiled plan that reaches the device or the launches, as bytes (fields
// one by one, so that struct padding does not enter).
static std::vector<unsigned char> plan_bytes(const CompileResult& cr) {
  std::vector<unsigned char> b;
  auto put = [&](const auto& x) {
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&x);
    b.insert(b.end(), p, p + sizeof(x));
  };
  for (const Step& s : cr.steps) {
    put(s.kind); put(s.pass.L); put(s.pass.c); put(s.pass.K); put(s.pass.st0); put(s.pass.nst);
    put(s.pass.flags); put(s.pass.swap_a); put(s.pass.swap_b); put(s.bytes); put(s.alu); put(s.dense_idx);
    for (int k = 0; k < s.pass.L; k++) put(s.pass.tpos[k]);
    for (int v : s.src_of) put(v);
  }
  for (const StageRec& st : cr.stages) {
    put(st.kind); put(st.op0); put(st.nops); put(st.rmask);
    for (int k = 0; k < 8; k++) put(st.rbits[k]);
  }
  for (const RegOp& r : cr.reg_ops) {
    put(r.type); put(r.s0); put(r.s1); put(r.tb); put(r.neg); put(r.csl); put(r.cot); put(r.mat);
    put(r.gmask); put(r.gbit);
  }
  for (const DevOp& d : cr.tile_ops) {
    put(d.type); put(d.k0); put(d.k1); put(d.nk); put(d.cmask); put(d.gmask); put(d.mat); put(d.gbit);
  }
  for (double v : cr.pool.f64) put(v);
  for (float v : cr.dense_w) put(v);
  return b;
}

// The compiler keeps working arrays per thread: the same circuit compiled on several threads
// at once, a few times each, must give the serial plan byte for byte.
static bool threads_consistent(int n, const std::vector<HGate>& gates, const std::vector<int>& sigma0,
                               const qs_compile_opts& o, const std::vector<unsigned char>& want, int nthreads) {
  std::vector<int> ok(nthreads, 1);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; t++)
    th.emplace_back([&, t] {
      for (int rep = 0; rep < 3; rep++) {
        CompileResult cr;
        std::string e;
        if (!compile_circuit(n, gates, sigma0, o, &cr, &e) || plan_bytes(cr) != want) ok[t] = 0;
      }
    });
  for (auto& x : th) x.join();
  for (int v : ok)
    if (!v) return false;
  return true;
}

static int euler_mode(const char* in, const char* out) {
  FILE* f = fopen(in, "rb");
  if (!f) return 2;
  int32_t count = 0;
  if (fread(&count, 4, 1, f) != 1) return 2;
  std::vector<double> m((size_t)count * 8);
  if (count && fread(m.data(), 8, m.size(), f) != m.size()) return 2;
  fclose(f);
  FILE* g = fopen(out, "wb");
  if (!g) return 2;
  for (int k = 0; k < count; k++) {
    C U[4], d1[4], rx[4], d2[4];
    for (int e = 0; e < 4; e++) U[e] = C(m[8 * k + 2 * e], m[8 * k + 2 * e + 1]);
    const int32_t okk = euler_split(U, d1, rx, d2) ? 1 : 0;
    fwrite(&okk, 4, 1, g);
    for (const C* fct : {d1, rx, d2})
      for (int e = 0; e < 4; e++) {
        const double re = fct[e].real(), im = fct[e].imag();
        fwrite(&re, 8, 1, g);
        fwrite(&im, 8, 1, g);
      }
  }
  fclose(g);
  return 0;
}

int main(int argc, char** argv) {
  if (argc == 4 && std::string(argv[1]) == "--euler") return euler_mode(argv[2], argv[3]);
  // optional: --threads T (also compile on T threads at once and compare the plans)
  int nthreads = 0;
  if (argc == 5 && std::string(argv[3]) == "--threads") {
    nthreads = atoi(argv[4]);
    argc = 3;
  }
  if (argc != 3) {
    fprintf(stderr, "usage: plan_emulator_host in.bin out.bin [--threads T] | --euler in.bin out.bin\n");
    return 2;
  }
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t n = 0, nops = 0;
  int64_t nmats = 0;
  qs_compile_opts o;
  int32_t has_cost = 0;
  qs_cost_model cost{};
  bool ok = fread(&n, 4, 1, f) == 1 && fread(&nops, 4, 1, f) == 1 && fread(&nmats, 8, 1, f) == 1 &&
            fread(&o, sizeof(o), 1, f) == 1 && fread(&has_cost, 4, 1, f) == 1 &&
            fread(&cost, sizeof(cost), 1, f) == 1;
  o.cost = has_cost ? &cost : nullptr;
  std::vector<qs_op> ops(nops);
  std::vector<double> mats(nmats > 0 ? nmats : 1);
  ok = ok && (nops == 0 || fread(ops.data(), sizeof(qs_op), nops, f) == (size_t)nops);
  ok = ok && (nmats == 0 || fread(mats.data(), 8, nmats, f) == (size_t)nmats);
  fclose(f);
  if (!ok) {
    fprintf(stderr, "bad input\n");
    return 2;
  }
  std::string err;
  if (!normalize_compile_opts(n, &o, &err)) {   // as qs_compile does
    fprintf(stderr, "options: %s\n", err.c_str());
    return 4;
  }
  std::vector<HGate> gates(nops);
  for (int i = 0; i < nops; i++)
    if (!make_hgate(n, ops[i], mats.data(), (size_t)nmats, &gates[i], &err)) {
      fprintf(stderr, "gate %d: %s\n", i, err.c_str());
      return 4;
    }
  std::vector<int> sigma0(n);
  for (int q = 0; q < n; q++) sigma0[q] = q;
  CompileResult cr;
  if (!compile_circuit(n, gates, sigma0, o, &cr, &err)) {
    fprintf(stderr, "compile: %s\n", err.c_str());
    return 4;
  }
  if (nthreads > 0)
    fprintf(stderr, "threads_consistent %d\n", threads_consistent(n, gates, sigma0, o, plan_bytes(cr), nthreads) ? 1 : 0);
  std::vector<C> psi(1ull << n, C(0, 0));
  psi[0] = 1;
  for (const Step& s : cr.steps) {
    switch (s.kind) {
      case ST_PASS: run_pass(psi, cr, s.pass); break;
      case ST_GATE: dev_op(psi, s.op, cr.pool, 0, false, false); break;
      case ST_PERMUTE: {
        std::vector<C> out(psi.size());
        for (uint64_t j = 0; j < psi.size(); j++) {
          uint64_t jn = 0;
          for (int p = 0; p < n; p++)
            if (bit(j, s.src_of[p])) jn |= 1ull << p;
          out[jn] = psi[j];
        }
        psi.swap(out);
        break;
      }
      case ST_DENSE: {   // the fused block on storage bits 0..5, as the compiler built it
        const C* U = &cr.dense_u[(size_t)s.dense_idx * 64 * 64];
        for (uint64_t row = 0; row < psi.size(); row += 64) {
          C x[64];
          for (int i = 0; i < 64; i++) x[i] = psi[row + i];
          for (int r = 0; r < 64; r++) {
            C acc(0, 0);
            for (int c = 0; c < 64; c++) acc += U[r * 64 + c] * x[c];
            psi[row + r] = acc;
          }
        }
        break;
      }
      case ST_RENORM: {
        double nrm = 0;
        for (const C& v : psi) nrm += std::norm(v);
        const double sc = 1.0 / std::sqrt(nrm);
        for (C& v : psi) v *= sc;
        break;
      }
      default:
        fprintf(stderr, "unknown step %d\n", s.kind);
        return 3;
    }
  }
  // the smallest scale any register op applies (the absorbed tangent-form factors make some
  // entries smaller than 1; the kernels need them well above the FP32 subnormal range)
  double min_scale = 1e300;
  for (const RegOp& r : cr.reg_ops) {
    if (r.type == OP_DTAB) {
      for (int j = 0; j < 32; j++)
        if ((r.csl >> j) & 1u) min_scale = std::min(min_scale, std::abs(entry(cr.pool, r.mat + j)));
    } else if (r.type == OP_RX) {
      const C e = entry(cr.pool, r.mat);
      min_scale = std::min(min_scale, std::max(std::fabs(e.real()), std::fabs(e.imag())));
    }
  }
  fprintf(stderr, "max_register_abs %.6e\nmin_register_scale %.6e\n", g_max_abs, min_scale);
  // the step sequence with the storage form each pass reads and writes (b = binary64,
  // d = double-float), for the test of the compiler's double-float storage rule
  fprintf(stderr, "steps");
  for (const Step& s : cr.steps) {
    switch (s.kind) {
      case ST_PASS:
        // P, form read, form written, "0" for a pass without stages, "s" for a pass whose
        // store carries a permutation (written out of place)
        fprintf(stderr, " P%c%c%s%s", (s.pass.flags & kPassInDF) ? 'd' : 'b', (s.pass.flags & kPassOutDF) ? 'd' : 'b',
                s.pass.nst == 0 ? "0" : "", s.pass.swap_a != s.pass.swap_b ? "s" : "");
        break;
      case ST_GATE: fprintf(stderr, " G"); break;
      case ST_PERMUTE: fprintf(stderr, " X"); break;
      case ST_RENORM: fprintf(stderr, " R"); break;
      case ST_DENSE: fprintf(stderr, " D"); break;
      default: fprintf(stderr, " ?"); break;
    }
  }
  fprintf(stderr, "\n");
  FILE* g = fopen(argv[2], "wb");
  if (!g) return 2;
  const int32_t nsteps = (int32_t)cr.steps.size();
  fwrite(&n, 4, 1, g);
  fwrite(&nsteps, 4, 1, g);
  for (int q = 0; q < n; q++) {
    const int32_t v = cr.sigma_final.empty() ? q : cr.sigma_final[q];
    fwrite(&v, 4, 1, g);
  }
  fwrite(psi.data(), sizeof(C), psi.size(), g);
  fclose(g);
  return 0;
}
