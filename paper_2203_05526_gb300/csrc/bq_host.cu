// Host side of the C ABI in include/bq.h: problem construction, the problem compiler
// (normal ordering and stencil tables of the coupled system, Eqs. 9a-c / 303a-c), the
// mapping of the measured operator (Eqs. 6, 10-13, 304), device layout, and stepping /
// evaluation drivers around the kernels of bq_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/bq.h"
#include "bq_internal.h"
#include "bq_launch.h"

using cplx = std::complex<double>;
using bq::ChanDesc;
using bq::EvalEntry;
using bq::EvalGroup;
using bq::InitEntry;
using bq::SysDesc;
using bq::TermDesc;
using bq::WorkItem;

// ---------------------------------------------------------------------------------------
// Errors.
// ---------------------------------------------------------------------------------------
static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(BQ_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));           \
  } while (0)

// ---------------------------------------------------------------------------------------
// Problem.
// ---------------------------------------------------------------------------------------
struct HTermH {
  cplx c;
  std::vector<int> u, v;
  int ch, conj, param;
};
struct JumpH {
  double rate;
  std::vector<cplx> c;
  std::vector<std::vector<int>> u, v;
};
struct ChannelH {
  int kind;
  std::vector<double> par;
};
struct SecularH {  // secular dissipator of one mode (Eq. 203 / Eq. S9)
  int mode;
  double kappa;
  std::vector<double> nbar;  // nbar[n]: occupation at the n <-> n+1 transition; 0 beyond
  double nb(int n) const { return n >= 0 && n < (int)nbar.size() ? nbar[n] : 0.0; }
};
using Key = std::pair<std::vector<int>, std::vector<int>>;

struct bq_problem {
  int nm = 0;
  std::vector<int> N;
  std::vector<HTermH> h;
  std::vector<JumpH> jumps;
  std::vector<SecularH> sec;
  std::vector<ChannelH> ch;
  std::vector<double> params;
  std::map<Key, cplx> measured, rho0;
  bool rho0_set = false;
};

static bool valid_powers(const bq_problem* p, const int* a) {
  for (int j = 0; j < p->nm; ++j)
    if (a[j] < 0 || a[j] > 16) return false;
  return true;
}

extern "C" int bq_problem_create(bq_problem** out, int n_modes, const int* fock_trunc) {
  if (!out) return fail(BQ_EINVAL, "out is NULL");
  if (n_modes < 1 || n_modes > BQ_MAX_MODES) return fail(BQ_EINVAL, "n_modes=%d outside 1..%d", n_modes, BQ_MAX_MODES);
  if (!fock_trunc) return fail(BQ_EINVAL, "fock_trunc is NULL");
  for (int j = 0; j < n_modes; ++j)
    if (fock_trunc[j] < 1 || fock_trunc[j] > 4096) return fail(BQ_EINVAL, "fock_trunc[%d]=%d", j, fock_trunc[j]);
  auto* p = new bq_problem();
  p->nm = n_modes;
  p->N.assign(fock_trunc, fock_trunc + n_modes);
  *out = p;
  return BQ_OK;
}

extern "C" void bq_problem_destroy(bq_problem* p) { delete p; }

extern "C" int bq_problem_add_channel(bq_problem* p, int kind, const double* params, int n_params, int* ch_out) {
  if (!p) return fail(BQ_EINVAL, "problem is NULL");
  static const int need[4] = {2, 4, 2, 3};
  if (kind < 0 || kind > 3) return fail(BQ_EINVAL, "unknown channel kind %d", kind);
  if (n_params < need[kind] || (n_params > 0 && !params)) return fail(BQ_EINVAL, "channel kind %d needs >= %d params", kind, need[kind]);
  if (kind == BQ_CH_PWC && (n_params % 2 != 0 || !(params[1] > 0.0)))
    return fail(BQ_EINVAL, "PWC channel needs (t_start, seg_len>0, re, im, ...)");
  if (kind == BQ_CH_GAUSS && !(params[3] > 0.0)) return fail(BQ_EINVAL, "GAUSS sigma must be > 0");
  p->ch.push_back({kind, std::vector<double>(params, params + n_params)});
  if (ch_out) *ch_out = (int)p->ch.size() - 1;
  return BQ_OK;
}

extern "C" int bq_problem_add_h_term(bq_problem* p, double re, double im, const int* u, const int* v, int channel,
                                     int conj, int param) {
  if (!p || !u || !v) return fail(BQ_EINVAL, "NULL argument");
  if (!valid_powers(p, u) || !valid_powers(p, v)) return fail(BQ_EINVAL, "monomial powers outside 0..16");
  if (channel < -1 || channel >= (int)p->ch.size()) return fail(BQ_EINVAL, "channel %d not defined", channel);
  if (param < -1) return fail(BQ_EINVAL, "param %d", param);
  p->h.push_back({cplx(re, im), std::vector<int>(u, u + p->nm), std::vector<int>(v, v + p->nm), channel,
                  channel < 0 ? 0 : (conj ? 1 : 0), param});
  return BQ_OK;
}

extern "C" int bq_problem_set_params(bq_problem* p, const double* values, int n) {
  if (!p || (n > 0 && !values) || n < 0) return fail(BQ_EINVAL, "bad params");
  p->params.assign(values, values + n);
  return BQ_OK;
}

extern "C" int bq_problem_add_jump(bq_problem* p, double kappa, int n_terms, const double* c_re, const double* c_im,
                                   const int* u, const int* v) {
  if (!p || n_terms < 1 || !c_re || !c_im || !u || !v) return fail(BQ_EINVAL, "bad jump arguments");
  if (!(kappa >= 0.0)) return fail(BQ_EINVAL, "jump rate must be >= 0");
  JumpH j;
  j.rate = kappa;
  for (int t = 0; t < n_terms; ++t) {
    if (!valid_powers(p, u + t * p->nm) || !valid_powers(p, v + t * p->nm))
      return fail(BQ_EINVAL, "jump monomial powers outside 0..16");
    j.c.push_back(cplx(c_re[t], c_im[t]));
    j.u.emplace_back(u + t * p->nm, u + (t + 1) * p->nm);
    j.v.emplace_back(v + t * p->nm, v + (t + 1) * p->nm);
  }
  p->jumps.push_back(std::move(j));
  return BQ_OK;
}

extern "C" int bq_problem_add_secular(bq_problem* p, int mode, double kappa, int n_nbar, const double* nbar) {
  if (!p) return fail(BQ_EINVAL, "problem is NULL");
  if (mode < 0 || mode >= p->nm) return fail(BQ_EINVAL, "mode %d outside 0..%d", mode, p->nm - 1);
  if (!(kappa >= 0.0)) return fail(BQ_EINVAL, "secular rate must be >= 0");
  if (n_nbar < 0 || (n_nbar > 0 && !nbar)) return fail(BQ_EINVAL, "bad nbar arguments");
  for (int n = 0; n < n_nbar; ++n)
    if (!(nbar[n] >= 0.0) || !std::isfinite(nbar[n])) return fail(BQ_EINVAL, "nbar[%d] must be finite and >= 0", n);
  p->sec.push_back({mode, kappa, std::vector<double>(nbar, nbar + n_nbar)});
  return BQ_OK;
}

static int set_elems(bq_problem* p, std::map<Key, cplx>& dst, int n, const int* k, const int* l, const double* re,
                     const double* im) {
  if (!p || n < 0 || (n > 0 && (!k || !l || !re || !im))) return fail(BQ_EINVAL, "bad element arguments");
  dst.clear();
  for (int i = 0; i < n; ++i) {
    std::vector<int> kk(k + i * p->nm, k + (i + 1) * p->nm), ll(l + i * p->nm, l + (i + 1) * p->nm);
    for (int j = 0; j < p->nm; ++j)
      if (kk[j] < 0 || ll[j] < 0) return fail(BQ_EINVAL, "negative Fock index");
    dst[{kk, ll}] += cplx(re[i], im[i]);
  }
  return BQ_OK;
}

extern "C" int bq_problem_set_measured(bq_problem* p, int n, const int* k, const int* l, const double* re,
                                       const double* im) {
  return set_elems(p, p->measured, n, k, l, re, im);
}

extern "C" int bq_problem_set_rho0(bq_problem* p, int n, const int* k, const int* l, const double* re,
                                   const double* im) {
  int r = set_elems(p, p->rho0, n, k, l, re, im);
  if (r == BQ_OK) p->rho0_set = true;
  return r;
}

// ---------------------------------------------------------------------------------------
// Normal ordering (S-eq. 103, r = 1): per mode
//   (a^dag)^p1 a^q1 (a^dag)^p2 a^q2 = sum_s s! C(q1,s) C(p2,s) (a^dag)^(p1+p2-s) a^(q1+q2-s).
// ---------------------------------------------------------------------------------------
using Poly = std::map<Key, cplx>;  // normal-ordered monomial -> coefficient

static double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}
static double fact(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

static Poly product(const Key& m1, const Key& m2, cplx c) {
  const int nm = (int)m1.first.size();
  Poly out;
  out[{std::vector<int>(nm, 0), std::vector<int>(nm, 0)}] = c;
  for (int j = 0; j < nm; ++j) {
    const int p1 = m1.first[j], q1 = m1.second[j], p2 = m2.first[j], q2 = m2.second[j];
    Poly next;
    for (auto& [key, val] : out) {
      for (int s = 0; s <= std::min(q1, p2); ++s) {
        const double w = fact(s) * binom(q1, s) * binom(p2, s);
        Key k2 = key;
        k2.first[j] = p1 + p2 - s;
        k2.second[j] = q1 + q2 - s;
        next[k2] += val * w;
      }
    }
    out.swap(next);
  }
  return out;
}

// ---------------------------------------------------------------------------------------
// Compiler.
// ---------------------------------------------------------------------------------------
struct RawTerm {
  int side;
  cplx c;
  cplx cb;  // coefficient with the parameter value set to 1
  int ch, conj, param;
  int a[BQ_MAXD], b[BQ_MAXD];
};

struct Compiled {
  int nm, M[BQ_MAX_MODES], method, basis, has_sep, has_r, r_diag = 0;
  int n_g, n_r;
  std::vector<TermDesc> terms;         // wtab offsets relative to this problem's weight block
  std::vector<double> wtab;            // weight tables
  std::vector<cplx> diag;              // 2*nm tables
  struct Sys {
    int p_flat, q_flat;
    cplx w, C;
    double gx0, gy0;          // stored values of x^p, y^q
    std::vector<cplx> vx, vy; // SVD initial conditions: stored G_x(0), G_y(0) (empty: monomial)
    std::vector<cplx> dC;     // d C / d theta_p (Eq. 304)
  };
  int n_params = 0;
  std::vector<Sys> sys;
  std::vector<std::pair<long long, cplx>> init;  // direct method: (R element offset, value)
  std::vector<EvalEntry> trace_entries;          // Tr(rho0 A) entries (kx, ly, factor)
  std::vector<EvalEntry> block_entries;          // lo=3 block (one per element)
  int block_dim;
  std::vector<ChanDesc> chans;
  std::vector<double> chpar;
  int halo_lo, halo_hi;
  double rho;                                    // spectral-radius bound for the stability check
};

static double s_of(int basis, int k) { return basis == BQ_BASIS_NUMBER ? std::sqrt(fact(k)) : 1.0; }

// weight of x^a d^b at index k on a grid of size M in the storage basis; 0 if out of grid
static double weight(int a, int b, int k, int M, int basis) {
  if (k < a) return 0.0;
  const int ks = k - a + b;
  if (ks >= M) return 0.0;
  double w = 1.0;
  for (int i = 1; i <= b; ++i) w *= (double)(k - a + i);  // (k-a+b)! / (k-a)!
  if (basis == BQ_BASIS_NUMBER) w *= std::sqrt(fact(k) / fact(ks));
  return w;
}

static double chan_max(const ChannelH& c) {
  switch (c.kind) {
    case BQ_CH_CONST: return std::abs(cplx(c.par[0], c.par[1]));
    case BQ_CH_GAUSS: return std::abs(cplx(c.par[0], c.par[1]));
    case BQ_CH_CEXP: return std::abs(cplx(c.par[0], c.par[1]));
    case BQ_CH_PWC: {
      double m = 0.0;
      for (size_t i = 2; i + 1 < c.par.size(); i += 2) m = std::max(m, std::abs(cplx(c.par[i], c.par[i + 1])));
      return m;
    }
  }
  return 0.0;
}

static int flat_index(const std::vector<int>& k, const int* M, int nm) {
  int f = 0;
  for (int j = 0; j < nm; ++j) f = f * M[j] + k[j];
  return f;
}

static int check_hermitian(const bq_problem* p) {
  // H = H^dag term by term: (c, u, v, ch, conj, param) pairs with (c*, v, u, ch, !conj, param).
  std::map<std::tuple<std::vector<int>, std::vector<int>, int, int, int>, cplx> m;
  for (auto& t : p->h) m[{t.u, t.v, t.ch, t.conj, t.param}] += t.c;
  for (auto& [key, c] : m) {
    auto& [u, v, ch, cj, par] = key;
    const int cj2 = ch < 0 ? 0 : 1 - cj;
    auto it = m.find({v, u, ch, cj2, par});
    const cplx c2 = it == m.end() ? cplx(0, 0) : it->second;
    if (std::abs(c - std::conj(c2)) > 1e-12 * std::max(1.0, std::abs(c)))
      return fail(BQ_EINVAL, "Hamiltonian is not Hermitian: add the conjugate of every term (swap u/v, conj channel)");
  }
  return BQ_OK;
}

// One-sided (Hestenes) Jacobi SVD of the n x n complex matrix W (column-major, overwritten):
// column rotations make W's columns orthogonal, W <- W V with V unitary (returned,
// column-major), so that the input equals W V^H and sigma_i = |W column i|.
static void jacobi_svd(int n, std::vector<cplx>& W, std::vector<cplx>& V) {
  V.assign((size_t)n * n, cplx(0, 0));
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 80; ++sweep) {
    double off = 0.0;
    for (int pc = 0; pc < n; ++pc)
      for (int qc = pc + 1; qc < n; ++qc) {
        cplx* a = &W[(size_t)pc * n];
        cplx* b = &W[(size_t)qc * n];
        double alpha = 0.0, beta = 0.0;
        cplx gamma(0, 0);
        for (int i = 0; i < n; ++i) {
          alpha += std::norm(a[i]);
          beta += std::norm(b[i]);
          gamma += std::conj(a[i]) * b[i];
        }
        const double g = std::abs(gamma);
        if (g == 0.0 || g <= 1e-15 * std::sqrt(alpha * beta)) continue;
        off = std::max(off, g / std::sqrt(alpha * beta));
        const cplx ph = std::conj(gamma / g);  // column q times ph makes a^H b real, = g
        const double zeta = (beta - alpha) / (2.0 * g);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::abs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        for (int i = 0; i < n; ++i) {
          const cplx ap = a[i], bq = b[i] * ph;
          a[i] = c * ap - sn * bq;
          b[i] = sn * ap + c * bq;
        }
        cplx* va = &V[(size_t)pc * n];
        cplx* vb = &V[(size_t)qc * n];
        for (int i = 0; i < n; ++i) {
          const cplx ap = va[i], bq = vb[i] * ph;
          va[i] = c * ap - sn * bq;
          vb[i] = sn * ap + c * bq;
        }
      }
    if (off < 1e-15) break;
  }
}

static int compile_problem(const bq_problem* p, const bq_map_opts& o, Compiled& C) {
  const int nm = p->nm;
  C.nm = nm;
  C.method = o.method;
  C.basis = o.basis != BQ_BASIS_AUTO ? o.basis
            : (o.method == BQ_METHOD_MAPPED && o.dtype == BQ_F64 ? BQ_BASIS_MONOMIAL : BQ_BASIS_NUMBER);
  if (o.method == BQ_METHOD_DIRECT) C.basis = BQ_BASIS_NUMBER;
  for (int j = 0; j < BQ_MAX_MODES; ++j) C.M[j] = 1;
  long long ng = 1;
  for (int j = 0; j < nm; ++j) {
    C.M[j] = o.grid[j] > 0 ? o.grid[j] : p->N[j];
    if (C.M[j] < 1 || C.M[j] > 127) return fail(BQ_EUNSUPPORTED, "grid M=%d per mode outside 1..127", C.M[j]);
    ng *= C.M[j];
  }
  if (ng * ng > (1LL << 30)) return fail(BQ_EUNSUPPORTED, "R too large");
  C.n_g = (int)ng;
  C.n_r = (int)(ng * ng);
  C.has_sep = o.method == BQ_METHOD_MAPPED ? 1 : 0;
  C.has_r = (o.method == BQ_METHOD_DIRECT || o.r_layout == BQ_R_FULL || o.r_layout == BQ_R_DIAG) ? 1 : 0;
  C.r_diag = (o.method == BQ_METHOD_MAPPED && o.r_layout == BQ_R_DIAG) ? 1 : 0;
  if (o.method == BQ_METHOD_DIRECT && o.r_layout == BQ_R_DIAG)
    return fail(BQ_EINVAL, "the diagonal residual layout applies to the mapped method only");
  for (auto& t : p->h)
    if (t.param >= (int)p->params.size()) return fail(BQ_EINVAL, "H term uses param %d but only %zu set", t.param, p->params.size());
  int r = check_hermitian(p);
  if (r != BQ_OK) return r;

  // ---- raw terms -----------------------------------------------------------------
  std::vector<RawTerm> raw;
  auto zero = [&](RawTerm& t) { for (int d = 0; d < BQ_MAXD; ++d) t.a[d] = t.b[d] = 0; };
  for (auto& t : p->h) {
    const cplx h = t.c * (t.param >= 0 ? p->params[t.param] : 1.0);
    RawTerm x; zero(x);
    x.side = bq::SIDE_X; x.c = cplx(0, 1) * h; x.cb = cplx(0, 1) * t.c; x.ch = t.ch; x.conj = t.conj; x.param = t.param;
    for (int j = 0; j < nm; ++j) { x.a[j] = t.u[j]; x.b[j] = t.v[j]; }
    raw.push_back(x);
    RawTerm y; zero(y);
    y.side = bq::SIDE_Y; y.c = cplx(0, -1) * h; y.cb = cplx(0, -1) * t.c; y.ch = t.ch; y.conj = t.conj; y.param = t.param;
    for (int j = 0; j < nm; ++j) { y.a[nm + j] = t.v[j]; y.b[nm + j] = t.u[j]; }
    raw.push_back(y);
  }
  for (auto& jp : p->jumps) {
    if (jp.rate == 0.0) continue;
    Poly LdL;
    for (size_t t = 0; t < jp.c.size(); ++t)
      for (size_t s = 0; s < jp.c.size(); ++s) {
        // L^dag L = sum_{t,s} conj(c_t) c_s m_t^dag m_s, m^dag = (a^dag)^v a^u
        Key mt_dag{jp.v[t], jp.u[t]}, ms{jp.u[s], jp.v[s]};
        for (auto& [k, v] : product(mt_dag, ms, std::conj(jp.c[t]) * jp.c[s])) LdL[k] += v;
        // sandwich kappa conj(c_t) c_s (m_t^dag)_left (m_s)_right
        RawTerm sw; zero(sw);
        sw.side = bq::SIDE_S; sw.c = jp.rate * std::conj(jp.c[t]) * jp.c[s]; sw.cb = sw.c; sw.ch = -1; sw.conj = 0; sw.param = -1;
        for (int j = 0; j < nm; ++j) {
          sw.a[j] = jp.v[t][j]; sw.b[j] = jp.u[t][j];            // left mult by m_t^dag
          sw.a[nm + j] = jp.v[s][j]; sw.b[nm + j] = jp.u[s][j];  // right mult by m_s
        }
        raw.push_back(sw);
      }
    for (auto& [k, v] : LdL) {
      if (v == cplx(0, 0)) continue;
      RawTerm x; zero(x);
      x.side = bq::SIDE_X; x.c = -0.5 * jp.rate * v; x.cb = x.c; x.ch = -1; x.conj = 0; x.param = -1;
      for (int j = 0; j < nm; ++j) { x.a[j] = k.first[j]; x.b[j] = k.second[j]; }
      raw.push_back(x);
      RawTerm y; zero(y);
      y.side = bq::SIDE_Y; y.c = -0.5 * jp.rate * v; y.cb = y.c; y.ch = -1; y.conj = 0; y.param = -1;
      for (int j = 0; j < nm; ++j) { y.a[nm + j] = k.second[j]; y.b[nm + j] = k.first[j]; }
      raw.push_back(y);
    }
  }

  // ---- fold static single-dimension diagonal terms; merge the rest -----------------
  const int ND = 2 * nm;
  int Md[BQ_MAXD];
  for (int d = 0; d < ND; ++d) Md[d] = C.M[d % nm];
  std::vector<int> doff(ND + 1, 0);
  for (int d = 0; d < ND; ++d) doff[d + 1] = doff[d] + Md[d];
  C.diag.assign(doff[ND], cplx(0, 0));
  std::map<std::tuple<int, int, int, int, std::vector<int>>, std::pair<cplx, cplx>> merged;  // (c, cb)
  for (auto& t : raw) {
    if (t.c == cplx(0, 0)) continue;
    bool diag = true;
    int nact = 0, dact = -1;
    for (int d = 0; d < ND; ++d) {
      if (t.a[d] != t.b[d]) diag = false;
      if (t.a[d] || t.b[d]) { ++nact; dact = d; }
    }
    if (t.side != bq::SIDE_S && t.ch < 0 && t.param < 0 && diag && nact <= 1) {
      const int d = nact == 0 ? (t.side == bq::SIDE_X ? 0 : nm) : dact;
      for (int k = 0; k < Md[d]; ++k) {
        double w = 1.0;
        for (int i = 0; i < t.a[d]; ++i) w *= (double)(k - i);  // k!/(k-a)!
        if (k < t.a[d]) w = 0.0;
        C.diag[doff[d] + k] += t.c * w;
      }
      continue;
    }
    std::vector<int> ab(2 * ND);
    for (int d = 0; d < ND; ++d) { ab[d] = t.a[d]; ab[ND + d] = t.b[d]; }
    auto& mv = merged[{t.side, t.ch, t.conj, t.param, ab}];
    mv.first += t.c;
    mv.second += t.cb;
  }
  if ((int)merged.size() > BQ_MAX_TERMS) return fail(BQ_EUNSUPPORTED, "%zu stencil terms > %d", merged.size(), BQ_MAX_TERMS);

  // strides: R index = kflat * n_g + lflat; flat = row-major over modes
  int stG[BQ_MAX_MODES] = {1, 1, 1, 1};
  for (int j = nm - 2; j >= 0; --j) stG[j] = stG[j + 1] * C.M[j + 1];
  int stR[BQ_MAXD];
  for (int j = 0; j < nm; ++j) { stR[j] = stG[j] * C.n_g; stR[nm + j] = stG[j]; }

  C.terms.clear();
  C.wtab.clear();
  C.halo_lo = C.halo_hi = 0;
  double rho_terms = 0.0;
  for (auto& [key, cc] : merged) {
    const cplx c = cc.first;
    if (c == cplx(0, 0) && cc.second == cplx(0, 0)) continue;
    auto& [side, ch, conj, param, ab] = key;
    if (!C.has_r && side == bq::SIDE_S) continue;  // sandwich acts only on R (and as its source)
    TermDesc td;
    std::memset(&td, 0, sizeof(td));
    td.c_re = c.real(); td.c_im = c.imag(); td.ch = ch; td.conj = conj; td.side = side; td.param = param;
    td.cb_re = cc.second.real(); td.cb_im = cc.second.imag();
    td.gslot_param = -1; td.gslot_pwc = -1;
    int nact = 0, dR = 0, dGx = 0, dGy = 0;
    double wmax_num = 1.0;
    for (int d = 0; d < ND; ++d) {
      const int a = ab[d], b = ab[ND + d];
      if (!a && !b) continue;
      td.dim[nact] = (int8_t)d;
      td.sh[nact] = (int8_t)(b - a);
      td.wtab[nact] = (int)C.wtab.size();
      double wm = 0.0;
      for (int k = 0; k < Md[d]; ++k) {
        C.wtab.push_back(weight(a, b, k, Md[d], C.basis));
        wm = std::max(wm, weight(a, b, k, Md[d], BQ_BASIS_NUMBER));
      }
      wmax_num *= wm;
      dR += (b - a) * stR[d];
      if (d < nm) dGx += (b - a) * stG[d]; else dGy += (b - a) * stG[d - nm];
      ++nact;
    }
    td.n_act = nact; td.deltaR = dR; td.deltaGx = dGx; td.deltaGy = dGy;
    C.halo_lo = std::max(C.halo_lo, std::abs(dR));  // symmetric: the adjoint gathers from p - delta
    C.halo_hi = C.halo_lo;
    C.terms.push_back(td);
    rho_terms += std::abs(c) * (ch >= 0 ? chan_max(p->ch[ch]) : 1.0) * wmax_num;
  }

  // ---- secular dissipators (Eq. 203 / Eq. S9) ---------------------------------------
  // In g_{k,l} the adjoint is a separable decay -kappa/2 [a(k_j) + a(l_j)],
  // a(m) = m (1 + nbar_{m-1}) + (m + 1) nbar_m, which joins the diagonal tables, plus two
  // jump terms restricted to k_j = l_j: g_{m,m} += kappa (1 + nbar_{m-1}) g_{m-1,m-1} and
  // g_{m,m} += kappa (m+1)^2 nbar_m g_{m+1,m+1} (the projector P of Eq. 302c / Eq. S15),
  // written as x y and d_x d_y stencils with diagonal-restricted sandwich terms.
  for (const SecularH& sh : p->sec) {
    if (sh.kappa == 0.0) continue;
    const int j = sh.mode, Mj = C.M[j];
    for (int m = 0; m < Mj; ++m) {
      const double a = m * (1.0 + sh.nb(m - 1)) + (m + 1) * sh.nb(m);
      C.diag[doff[j] + m] += -0.5 * sh.kappa * a;
      C.diag[doff[nm + j] + m] += -0.5 * sh.kappa * a;
    }
    if (!C.has_r) continue;
    bool any_up = false;
    for (int m = 0; m + 1 < Mj; ++m) any_up = any_up || sh.nb(m) > 0.0;
    for (int dir = 0; dir < (any_up ? 2 : 1); ++dir) {  // 0: source m-1 (x y), 1: source m+1 (d_x d_y)
      const int a = dir == 0 ? 1 : 0, b = dir == 0 ? 0 : 1;
      TermDesc td;
      std::memset(&td, 0, sizeof(td));
      td.c_re = 1.0; td.cb_re = 1.0; td.ch = -1; td.side = bq::SIDE_S; td.param = -1;
      td.gslot_param = -1; td.gslot_pwc = -1;
      td.n_act = 2;
      td.diagp1 = (int8_t)(j + 1);
      td.dim[0] = (int8_t)j; td.dim[1] = (int8_t)(nm + j);
      td.sh[0] = td.sh[1] = (int8_t)(b - a);
      double wmax = 0.0;
      td.wtab[0] = (int)C.wtab.size();
      for (int m = 0; m < Mj; ++m) {
        const double rate = dir == 0 ? sh.kappa * (1.0 + sh.nb(m - 1)) : sh.kappa * sh.nb(m);
        C.wtab.push_back(rate * weight(a, b, m, Mj, C.basis));
        wmax = std::max(wmax, rate * weight(a, b, m, Mj, BQ_BASIS_NUMBER) * weight(a, b, m, Mj, BQ_BASIS_NUMBER));
      }
      td.wtab[1] = (int)C.wtab.size();
      for (int l = 0; l < Mj; ++l) C.wtab.push_back(weight(a, b, l, Mj, C.basis));
      td.deltaR = (b - a) * (stR[j] + stR[nm + j]);
      td.deltaGx = (b - a) * stG[j];
      td.deltaGy = (b - a) * stG[j];
      C.halo_lo = std::max(C.halo_lo, std::abs(td.deltaR));
      C.halo_hi = C.halo_lo;
      C.terms.push_back(td);
      rho_terms += wmax;
    }
  }
  if ((int)C.terms.size() > BQ_MAX_TERMS) return fail(BQ_EUNSUPPORTED, "%zu stencil terms > %d", C.terms.size(), BQ_MAX_TERMS);

  // ---- stability bound: max |diag| over the grid + sum of off-diagonal magnitudes ----
  {
    double dmax = 0.0;
    const int npts = C.has_r ? C.n_r : C.n_g;
    const int nd = C.has_r ? ND : nm;
    std::vector<int> idx(ND, 0);
    for (int pnt = 0; pnt < npts; ++pnt) {
      int rr = pnt;
      for (int d = nd - 1; d >= 0; --d) { idx[d] = rr % Md[d]; rr /= Md[d]; }
      cplx s(0, 0);
      for (int d = 0; d < nd; ++d) s += C.diag[doff[d] + idx[d]];
      dmax = std::max(dmax, std::abs(s));
      if (!C.has_r) {  // G_y too
        cplx s2(0, 0);
        for (int d = 0; d < nm; ++d) s2 += C.diag[doff[nm + d] + idx[d]];
        dmax = std::max(dmax, std::abs(s2));
      }
    }
    C.rho = dmax + rho_terms;
  }
  // diagonal residual layout: R holds its k = l entries only (index = flat k); a term
  // contributes an R source only if it shifts x and y alike, at offset deltaGx
  if (C.r_diag) {
    C.n_r = C.n_g;
    C.halo_lo = 0;
    for (const TermDesc& td : C.terms)
      if (td.deltaGx == td.deltaGy) C.halo_lo = std::max(C.halo_lo, std::abs(td.deltaGx));
    C.halo_hi = C.halo_lo;
  }

  C.n_params = (int)p->params.size();
  // ---- channels ----------------------------------------------------------------------
  C.chans.clear(); C.chpar.clear();
  for (auto& ch : p->ch) {
    ChanDesc cd;
    cd.kind = ch.kind; cd.n_par = (int)ch.par.size(); cd.par_off = (int)C.chpar.size(); cd.pad = 0;
    C.chans.push_back(cd);
    C.chpar.insert(C.chpar.end(), ch.par.begin(), ch.par.end());
  }

  // ---- systems (initial conditions, Eqs. 10 / 13) -----------------------------------
  // om_j, eta_j of Eq. 304: static coefficients of a_j^dag a_j and a_j^dag^2 a_j^2.
  std::vector<double> om(nm, 0.0), et(nm, 0.0);
  for (auto& t : p->h) {
    if (t.ch >= 0) continue;
    int nz = 0, j0 = -1;
    for (int j = 0; j < nm; ++j) if (t.u[j] || t.v[j]) { ++nz; j0 = j; }
    if (nz != 1) continue;
    const double cr = (t.c * (t.param >= 0 ? p->params[t.param] : 1.0)).real();
    if (t.u[j0] == 1 && t.v[j0] == 1) om[j0] += cr;
    if (t.u[j0] == 2 && t.v[j0] == 2) et[j0] += cr;
  }
  C.sys.clear(); C.init.clear();
  auto in_grid = [&](const std::vector<int>& k) {
    for (int j = 0; j < nm; ++j) if (k[j] >= C.M[j]) return false;
    return true;
  };
  auto sfl = [&](const std::vector<int>& k) {  // s(k) of the storage basis (product over modes)
    double s = 1.0;
    for (int j = 0; j < nm; ++j) s *= s_of(C.basis, k[j]);
    return s;
  };
  auto sqfact = [&](const std::vector<int>& k) {
    double s = 1.0;
    for (int j = 0; j < nm; ++j) s *= std::sqrt(fact(k[j]));
    return s;
  };
  if (C.method == BQ_METHOD_DIRECT) {
    C.sys.push_back({0, 0, cplx(1, 0), cplx(0, 0), 0.0, 0.0, std::vector<cplx>(p->params.size(), cplx(0, 0))});
    for (auto& [kl, v] : p->measured)
      if (in_grid(kl.first) && in_grid(kl.second) && v != cplx(0, 0))
        C.init.push_back({(long long)flat_index(kl.first, C.M, nm) * C.n_g + flat_index(kl.second, C.M, nm), v});
  } else if (o.ic_mode == BQ_IC_SVD) {
    // g(0) in the storage basis (stored value s(p) s(q) <p|A|q> / sqrt(p! q!)), factored as
    // sum_i sigma_i u_i v_i^H; one system per sigma_i > 1e-12 sigma_max
    const int n = C.n_g;
    if (n > 1024) return fail(BQ_EUNSUPPORTED, "SVD initial conditions need prod M <= 1024 (%d)", n);
    std::vector<cplx> W((size_t)n * n, cplx(0, 0)), V;
    for (auto& [kl, v] : p->measured) {
      if (!in_grid(kl.first) || !in_grid(kl.second) || v == cplx(0, 0)) continue;
      const int pf = flat_index(kl.first, C.M, nm), qf = flat_index(kl.second, C.M, nm);
      W[(size_t)qf * n + pf] += v / sqfact(kl.first) / sqfact(kl.second) * sfl(kl.first) * sfl(kl.second);
    }
    jacobi_svd(n, W, V);
    std::vector<std::pair<double, int>> sig;
    double smax = 0.0;
    for (int i = 0; i < n; ++i) {
      double s2 = 0.0;
      for (int k = 0; k < n; ++k) s2 += std::norm(W[(size_t)i * n + k]);
      sig.push_back({-std::sqrt(s2), i});
      smax = std::max(smax, std::sqrt(s2));
    }
    std::sort(sig.begin(), sig.end());
    for (auto& [ns, i] : sig) {
      if (!(-ns > 1e-12 * smax)) break;
      Compiled::Sys s;
      s.p_flat = -1; s.q_flat = -1;
      s.w = cplx(1, 0);
      s.C = cplx(0, 0);
      s.dC.assign(p->params.size(), cplx(0, 0));
      s.gx0 = s.gy0 = 0.0;
      s.vx.assign(W.begin() + (size_t)i * n, W.begin() + (size_t)(i + 1) * n);
      s.vy.resize(n);
      for (int k = 0; k < n; ++k) s.vy[k] = std::conj(V[(size_t)i * n + k]);
      C.sys.push_back(s);
    }
  } else {
    for (auto& [kl, v] : p->measured) {
      if (!in_grid(kl.first) || !in_grid(kl.second) || v == cplx(0, 0)) continue;
      Compiled::Sys s;
      s.p_flat = flat_index(kl.first, C.M, nm);
      s.q_flat = flat_index(kl.second, C.M, nm);
      s.w = v / sqfact(kl.first) / sqfact(kl.second);  // g_{p,q}(0) = <p|A|q>/sqrt(p! q!)
      double cs = 0.0;
      for (int j = 0; j < nm; ++j) {
        const int pj = kl.first[j], qj = kl.second[j];
        cs += (om[j] - et[j]) * (pj + qj) + et[j] * (pj * pj + qj * qj);
      }
      s.C = o.c_mode == BQ_C_ZERO ? cplx(0, 0) : cplx(0, -0.5 * cs);
      s.dC.assign(p->params.size(), cplx(0, 0));
      if (o.c_mode != BQ_C_ZERO) {
        for (auto& t : p->h) {
          if (t.param < 0 || t.ch >= 0) continue;
          int nz = 0, j0 = -1;
          for (int j = 0; j < nm; ++j) if (t.u[j] || t.v[j]) { ++nz; j0 = j; }
          if (nz != 1) continue;
          const double cr = t.c.real();
          const int pj = kl.first[j0], qj = kl.second[j0];
          if (t.u[j0] == 1 && t.v[j0] == 1) s.dC[t.param] += cplx(0, -0.5 * cr * (pj + qj));
          if (t.u[j0] == 2 && t.v[j0] == 2) s.dC[t.param] += cplx(0, -0.5 * cr * (pj * pj + qj * qj - pj - qj));
        }
      }
      // G_x = x^p, G_y = y^q in the storage basis (values s(p), s(q)); R = 0
      s.gx0 = sfl(kl.first);
      s.gy0 = sfl(kl.second);
      C.sys.push_back(s);
    }
  }

  // ---- evaluation entries -----------------------------------------------------------
  auto unflat = [&](int f) {
    std::vector<int> k(nm);
    for (int j = nm - 1; j >= 0; --j) { k[j] = f % C.M[j]; f /= C.M[j]; }
    return k;
  };
  auto factor = [&](int kx, int ly) {  // A_{k,l} = sqrt(k! l!) / (s(k) s(l)) * stored value
    const auto k = unflat(kx), l = unflat(ly);
    return sqfact(k) * sqfact(l) / (sfl(k) * sfl(l));
  };
  C.trace_entries.clear();
  std::map<Key, cplx> rho0 = p->rho0;
  if (!p->rho0_set) rho0[{std::vector<int>(nm, 0), std::vector<int>(nm, 0)}] = cplx(1, 0);
  for (auto& [kl, r0] : rho0) {
    // Tr(rho0 A) = sum <k|rho0|l> <l|A|k>
    if (!in_grid(kl.first) || !in_grid(kl.second) || r0 == cplx(0, 0)) continue;
    EvalEntry e;
    std::memset(&e, 0, sizeof(e));
    e.kx = flat_index(kl.second, C.M, nm);
    e.ly = flat_index(kl.first, C.M, nm);
    const cplx f = r0 * factor(e.kx, e.ly);
    e.f_re = f.real(); e.f_im = f.imag();
    C.trace_entries.push_back(e);
  }
  int lo[BQ_MAX_MODES] = {1, 1, 1, 1};
  int D = 1;
  for (int j = 0; j < nm; ++j) { lo[j] = std::min(3, C.M[j]); D *= lo[j]; }
  C.block_dim = D;
  C.block_entries.clear();
  for (int a = 0; a < D; ++a)
    for (int b = 0; b < D; ++b) {
      std::vector<int> k(nm), l(nm);
      int ra = a, rb = b;
      for (int j = nm - 1; j >= 0; --j) { k[j] = ra % lo[j]; ra /= lo[j]; l[j] = rb % lo[j]; rb /= lo[j]; }
      EvalEntry e;
      std::memset(&e, 0, sizeof(e));
      e.kx = flat_index(k, C.M, nm);
      e.ly = flat_index(l, C.M, nm);
      e.f_re = factor(e.kx, e.ly); e.f_im = 0.0;
      C.block_entries.push_back(e);
    }
  return BQ_OK;
}

// ---------------------------------------------------------------------------------------
// State.
// ---------------------------------------------------------------------------------------
struct Layout {
  size_t off_sys, off_terms, off_chans, off_chpar, off_work, off_m1, off_order, off_dc, off_pparams, off_precs, off_obs, off_groups, off_entries, off_out, off_wtab, off_diag,
      off_ctrl, off_init, off_y, off_comp, off_ua, off_ub, off_acc, total;
};

struct bq_state {
  int B = 0, nm = 0, dtype = 0, method = 0, basis = 0, n_sys = 0, n_work = 0, smem_bytes = 0, use_m1 = 0, m1_variant = 0;
  int trace_small = 0, block_small = 0;
  int solve_ok = 0, solve_smem = 0, last_solve_grid = 0, solve_mg = 0, solve_mg_smem = 0;
  int solve_via_step = 0;  // bq_solve runs bq_step (BQ_SOLVE_STEP)
  int use_pipe = 0, pipe_off_u = 0, pipe_zero_off = 0, pipe_zero_bytes = 0, pipe_mmax = 0, pipe_obs = 0;
  int pipe_slot[4] = {0, 0, 0, 0}, pipe_nslots[4] = {2, 2, 2, 2}, pipe_grid[4] = {1, 1, 1, 1}, pipe_mv_bytes = 0;
  // one launch for all steps of a bq_step call (k_steps_pipe): enabled, and its grid (0: does
  // not fit)
  int pipe_fused = 1, pipe_steps_grid = 0;
  // 1 after bq_load_state: comp is zero by definition but not written yet (the pipelined and
  // streaming kernels skip reading it at their next stage 1; every other consumer clears it
  // first, see ensure_comp)
  int comp_zero = 0;
  // 1 while the per-system Tr(rho0 A) contributions the pipelined kernel's last stage 4 left
  // in the pool describe the current state (bq_evaluate then only reads them back)
  int obs_valid = 0;
  int has_diag = 0;     // some term acts only on diagonal index pairs (secular dissipator)
  int r_diag = 0;       // diagonal residual layout
  int has_gread = 0;    // some work item reads its R sources from global memory
  int work_cap = 0, tile = 0;  // work-item capacity of the pool; tiled schedule (0 = default)
  int gread_sched = 0;         // split tiles read R from global memory (schedule)
  double tune_grad_us = 0.0;   // last bq_autotune_grad result
  int lanes = 1;               // lanes per point of the tiled forward and the adjoint stage kernels
  int grad_coop = 1;           // bq_grad: cooperative segment kernels where available
  int ng_max = 0;      // largest G_x / G_y point count over the systems
  // schedules (bq_get_tune / bq_set_tune / bq_autotune)
  int pipe_ok = 0;      // the pipelined path is available (single mode, two slots fit)
  int pipe_cap = 0;     // resident pipelined CTAs per SM (0 = occupancy limit)
  int solve_mg_ok = 0;  // the merged-stencil persistent solve is available
  int solve_cap = 0;    // resident persistent-solve CTAs per SM (0 = occupancy limit)
  int tune_n = 0;
  double tune_step_us = 0.0, tune_solve_us = 0.0;
  int grad_size = 0, adj_smem = 0, srcred_stride = 0, max_s = 0;
  std::vector<TermDesc> terms_host;
  std::vector<ChanDesc> chans_host;
  std::vector<double> chpar_host;
  int n_trace_groups = 0, n_block_groups = 0, block_dim = 0;
  int64_t total_elems = 0;
  double dt_max = 0.0, horizon = 0.0, tau = 0.0;
  int reverse = 1;
  char* pool = nullptr;
  Layout L{};
  std::vector<SysDesc> sys;
  std::vector<int> prob_M;  // B * BQ_MAX_MODES
  // tau control (host mirror) and graph cache
  double tau_base_host = 0.0;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t grad_stream[2] = {nullptr, nullptr};  // bq_grad: segment recomputation, backward sweep
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0.0;
  int graph_steps = 0;
};

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct Plan {
  std::vector<Compiled> comp;
  std::vector<SysDesc> sys;
  std::vector<TermDesc> terms;
  std::vector<ChanDesc> chans;
  std::vector<double> chpar;
  std::vector<WorkItem> work;
  std::vector<EvalGroup> groups;
  std::vector<EvalEntry> entries;
  std::vector<double> wtab;
  std::vector<cplx> diag;
  std::vector<InitEntry> init;
  int n_trace_groups = 0, n_block_groups = 0, block_dim = 0, smem_bytes = 0;
  int use_m1 = 0;  // single-mode fast path: one CTA per system, whole system in shared memory
  int m1_variant = 0;
  std::vector<bq::M1Sys> m1;
  std::vector<int> order;  // batched solve queue (largest system first); empty: not eligible
  // pipelined stage kernel
  int use_pipe = 0, pipe_off_u = 0, pipe_zero_off = 0, pipe_zero_bytes = 0, pipe_slot = 0, pipe_mmax = 0;
  int pipe_obs = 1;  // the last stage evaluates every problem's Tr(rho0 A) (supports of <= 32 entries)
  std::vector<unsigned char> pparams;
  std::vector<bq::PipeRec> precs;
  size_t work_cap = 0;  // work-item capacity of the pool (the smallest schedulable tile, 32 points)
  int solve_smem = 0;
  int solve_mg = 0, solve_mg_smem = 0;  // merged-stencil persistent solve
  int adj_smem = 0;  // shared memory of the adjoint stage kernel
  int srcred_stride = 0, max_s = 0;
  std::vector<int> wbase;  // per problem: offset of its weight tables in the pool
  std::vector<int> grad_offs;  // per problem: first gradient slot
  std::vector<cplx> dc;        // d C / d theta per system and parameter
  int grad_size = 0;
  int64_t total_elems = 0;
  double rho = 0.0, dt_max = 0.0;
  Layout L{};
};

// Work items of the tiled stage kernel.  A system that fits in one shared-memory tile takes
// one CTA (R, G_x and G_y) unless the batch is too small to fill the GPU that way; larger ones
// are split into tiles of R with halo windows (or, when the halo does not fit beside a tile,
// tiles that read R from global memory) and items that update chunks of [G_x | G_y].
// tile > 0 sets the length of the split tiles (a schedule); 0 = enough tiles for two CTAs
// per SM.  force_gread: split tiles read R from global memory (L1 / L2) instead of staging a
// halo window (a schedule: less shared memory per CTA, no staging phase).  smem_max / adj_max: complex elements of shared memory of the forward and the
// adjoint stage kernel.
#define BQ_SEP_CHUNK 64

// Lanes per point of the tiled kernels: enough threads for about half the GPU's warp slots
// (152 SMs x 16 warps), with up to four lanes sharing the terms of a point when the launch
// has fewer points than that.
static int default_lanes(const std::vector<SysDesc>& sys) {
  int64_t pts = 0;
  for (const SysDesc& sd : sys) pts += (sd.has_r ? sd.n_r : 0) + (sd.has_sep ? 2 * sd.n_g : 0);
  const int64_t half = 152 * 16 * 32;
  return pts >= half ? 1 : (pts >= half / 2 ? 2 : 4);
}
static void build_work(const std::vector<SysDesc>& sys, size_t cs, int tile, int force_gread,
                       std::vector<WorkItem>& work, int& smem_max, int& adj_max) {
  const int budget = (int)(96 * 1024 / cs);
  work.clear();
  smem_max = adj_max = 0;
  const int nsys = (int)sys.size();
  for (int i = 0; i < nsys; ++i) {
    const SysDesc& sd = sys[i];
    const int sep = (sd.has_sep ? 2 * sd.n_g : 0) + sd.cw_elems;  // G_x, G_y and the forward kernel's tables
    const int adj_sep = sd.has_sep ? (2 + 2 * sd.n_sterms) * sd.n_g : 0;
    const int nsep = sd.has_sep ? 2 * sd.n_g : 0;
    if (!sd.has_r) {
      // separable part only: one CTA per system, or chunks of it (the tile length, else
      // BQ_SEP_CHUNK points) when the batch is too small to fill the GPU with systems
      const int chunk = nsys < 2 * 152 ? (tile > 0 ? tile : BQ_SEP_CHUNK) : std::max(nsep, 1);
      for (int g0 = 0; g0 < std::max(nsep, 1); g0 += chunk)
        work.push_back(WorkItem{i, 0, 0, g0, std::min(nsep, g0 + chunk), 0, 0, sep, 0});
      smem_max = std::max(smem_max, sep);
      adj_max = std::max(adj_max, adj_sep);
      continue;
    }
    // too few systems to fill the GPU with one CTA each: split those with a few hundred points
    const bool few = nsys < 2 * 152 && sd.n_r + nsep >= 2 * 128;
    if (sd.n_r + sep <= budget && !few) {
      work.push_back(WorkItem{i, 0, sd.n_r, 0, nsep, 0, sd.n_r, sd.n_r + sep, 0});
      smem_max = std::max(smem_max, sd.n_r + sep);
      adj_max = std::max(adj_max, sd.n_r + adj_sep);
      continue;
    }
    int tl = budget - sep - sd.halo_lo - sd.halo_hi;
    // the halo does not fit next to a tile (or the schedule asks for it): read R from global memory
    const int gread = (tl < 64 || force_gread) ? 1 : 0;
    if (gread) tl = 1 << 30;
    if (tile > 0) {
      tl = gread ? tile : std::min(tl, tile);
    } else {
      // enough CTAs per launch to occupy every SM twice
      const int want_tiles = std::max(1, (2 * 152 + nsys - 1) / nsys);
      const int tl_par = std::max(few ? 256 : 64, (sd.n_r + want_tiles - 1) / want_tiles);
      tl = std::min(tl, tl_par);
    }
    // the separable part of a split system: items of its own (the tile length, else
    // BQ_SEP_CHUNK points each)
    const int chunk = tile > 0 ? tile : BQ_SEP_CHUNK;
    for (int g0 = 0; g0 < nsep; g0 += chunk) {
      work.push_back(WorkItem{i, 0, 0, g0, std::min(nsep, g0 + chunk), 0, 0, sep, 0});
      smem_max = std::max(smem_max, sep);
      adj_max = std::max(adj_max, adj_sep);
    }
    for (int s0 = 0; s0 < sd.n_r; s0 += tl) {
      WorkItem w;
      w.sys = i; w.start = s0; w.len = std::min(tl, sd.n_r - s0); w.sep_lo = w.sep_hi = 0;
      w.win_lo = gread ? s0 : std::max(0, s0 - sd.halo_lo);
      w.win_hi = gread ? s0 : std::min(sd.n_r, s0 + w.len + sd.halo_hi);
      w.smem_elems = (w.win_hi - w.win_lo) + sep; w.gread = gread;
      smem_max = std::max(smem_max, w.smem_elems);
      adj_max = std::max(adj_max, (w.win_hi - w.win_lo) + adj_sep);
      work.push_back(w);
    }
  }
}

static int make_plan(const bq_problem* const* probs, int B, const bq_map_opts* o, Plan& P) {
  if (!probs || B < 1 || !o) return fail(BQ_EINVAL, "bad map arguments");
  if (o->method != BQ_METHOD_MAPPED && o->method != BQ_METHOD_DIRECT) return fail(BQ_EINVAL, "method");
  if (o->dtype != BQ_F64 && o->dtype != BQ_F32) return fail(BQ_EINVAL, "dtype");
  if (o->r_layout != BQ_R_FULL && o->r_layout != BQ_R_OFF && o->r_layout != BQ_R_DIAG) return fail(BQ_EINVAL, "r_layout");
  if (o->ic_mode != BQ_IC_MONOMIAL && o->ic_mode != BQ_IC_SVD) return fail(BQ_EINVAL, "ic_mode");
  const int nm = probs[0] ? probs[0]->nm : 0;
  const size_t cs = o->dtype == BQ_F64 ? 16 : 8;  // complex element size
  const size_t rs = cs / 2;
  P.comp.resize(B);
  int64_t elem = 0;
  for (int b = 0; b < B; ++b) {
    if (!probs[b]) return fail(BQ_EINVAL, "problem %d is NULL", b);
    if (probs[b]->nm != nm) return fail(BQ_EINVAL, "all problems of a batch need the same number of modes");
    int r = compile_problem(probs[b], *o, P.comp[b]);
    if (r != BQ_OK) return r;
    Compiled& C = P.comp[b];
    if (C.sys.empty()) return fail(BQ_EINVAL, "problem %d: measured operator is zero on the grid", b);
    P.rho = std::max(P.rho, C.rho);
    const int term_off = (int)P.terms.size();
    const int wbase = (int)P.wtab.size();
    P.wbase.push_back(wbase);
    // gradient layout of this problem: [theta_0 .. theta_{P-1} | (Re, Im) of every segment of
    // every piecewise-constant channel, channels in order]
    const int grad_off = P.grad_size;
    std::vector<int> pwc_off(C.chans.size(), -1);
    int gsz = C.n_params;
    for (size_t c = 0; c < C.chans.size(); ++c)
      if (C.chans[c].kind == BQ_CH_PWC) { pwc_off[c] = gsz; gsz += 2 * ((C.chans[c].n_par - 2) / 2); }
    P.grad_size += gsz;
    P.grad_offs.push_back(grad_off);
    for (auto td : C.terms) {
      td.gslot_param = td.param >= 0 ? grad_off + td.param : -1;
      td.gslot_pwc = (td.ch >= 0 && pwc_off[td.ch] >= 0) ? grad_off + pwc_off[td.ch] : -1;
      for (int i = 0; i < td.n_act; ++i) td.wtab[i] += wbase;
      if (td.ch >= 0) td.ch += (int)P.chans.size();
      P.terms.push_back(td);
    }
    P.wtab.insert(P.wtab.end(), C.wtab.begin(), C.wtab.end());
    const int cbase = (int)P.chpar.size();
    for (auto cd : C.chans) { cd.par_off += cbase; P.chans.push_back(cd); }
    P.chpar.insert(P.chpar.end(), C.chpar.begin(), C.chpar.end());
    const int diag_off = (int)P.diag.size();
    P.diag.insert(P.diag.end(), C.diag.begin(), C.diag.end());
    const int sys_off = (int)P.sys.size();
    for (auto& s : C.sys) {
      SysDesc sd;
      std::memset(&sd, 0, sizeof(sd));
      sd.prob = b; sd.nm = nm;
      for (int j = 0; j < BQ_MAX_MODES; ++j) sd.M[j] = C.M[j];
      sd.has_sep = C.has_sep; sd.has_r = C.has_r; sd.n_g = C.n_g; sd.n_r = C.n_r; sd.r_diag = C.r_diag;
      sd.term_off = term_off; sd.n_terms = (int)C.terms.size(); sd.diag_off = diag_off;
      sd.halo_lo = C.halo_lo; sd.halo_hi = C.halo_hi; sd.p_flat = s.p_flat; sd.q_flat = s.q_flat;
      int stG[BQ_MAX_MODES] = {1, 1, 1, 1};
      for (int j = nm - 2; j >= 0; --j) stG[j] = stG[j + 1] * C.M[j + 1];
      for (int j = 0; j < nm; ++j) { sd.stG[j] = stG[j]; sd.stR[j] = stG[j] * C.n_g; sd.stR[nm + j] = stG[j]; }
      sd.off_gx = sd.off_gy = sd.off_r = -1;
      // element layout of one system: [G_x | G_y | R], each block 4-element aligned (32 bytes
      // in FP32: whole DRAM sectors, and 16-byte aligned bulk copies in either precision)
      auto pad4 = [](int64_t x) { return (x + 3) & ~(int64_t)3; };
      if (C.has_sep) { sd.off_gx = elem; elem += pad4(C.n_g); sd.off_gy = elem; elem += pad4(C.n_g); }
      if (C.has_r) { sd.off_r = elem; elem += pad4(C.n_r); }
      sd.c_re = s.C.real(); sd.c_im = s.C.imag(); sd.w_re = s.w.real(); sd.w_im = s.w.imag();
      sd.n_params = C.n_params;
      sd.grad_off = grad_off;
      sd.dc_off = (int)P.dc.size();
      P.dc.insert(P.dc.end(), s.dC.begin(), s.dC.end());
      P.sys.push_back(sd);
    }
    // initial values
    if (C.method == BQ_METHOD_DIRECT) {
      for (auto& [off, v] : C.init) P.init.push_back({P.sys[sys_off].off_r + off, v.real(), v.imag()});
    } else {
      for (size_t i = 0; i < C.sys.size(); ++i) {
        const SysDesc& sd = P.sys[sys_off + i];
        if (!C.sys[i].vx.empty()) {  // SVD initial condition: whole vectors
          for (int k = 0; k < C.n_g; ++k) {
            const cplx a = C.sys[i].vx[k], b = C.sys[i].vy[k];
            if (a != cplx(0, 0)) P.init.push_back({sd.off_gx + k, a.real(), a.imag()});
            if (b != cplx(0, 0)) P.init.push_back({sd.off_gy + k, b.real(), b.imag()});
          }
        } else {
          P.init.push_back({sd.off_gx + C.sys[i].p_flat, C.sys[i].gx0, 0.0});
          P.init.push_back({sd.off_gy + C.sys[i].q_flat, C.sys[i].gy0, 0.0});
        }
      }
    }
    // evaluation groups: trace group b, then block groups appended later
    EvalGroup g;
    std::memset(&g, 0, sizeof(g));
    g.prob = b; g.e_off = (int)P.entries.size(); g.n_e = (int)C.trace_entries.size();
    g.sys_off = sys_off; g.n_sys = (int)C.sys.size();
    P.entries.insert(P.entries.end(), C.trace_entries.begin(), C.trace_entries.end());
    P.groups.push_back(g);
  }
  P.n_trace_groups = B;
  P.block_dim = P.comp[0].block_dim;
  for (int b = 0; b < B; ++b) {
    const Compiled& C = P.comp[b];
    if (C.block_dim != P.block_dim) { P.block_dim = -1; break; }
  }
  if (P.block_dim > 0) {
    int sys_off = 0;
    for (int b = 0; b < B; ++b) {
      const Compiled& C = P.comp[b];
      for (auto& e : C.block_entries) {
        EvalGroup g;
        std::memset(&g, 0, sizeof(g));
        g.prob = b; g.e_off = (int)P.entries.size(); g.n_e = 1; g.sys_off = sys_off; g.n_sys = (int)C.sys.size();
        P.entries.push_back(e);
        P.groups.push_back(g);
      }
      sys_off += (int)C.sys.size();
    }
    P.n_block_groups = (int)P.groups.size() - B;
  }
  P.total_elems = std::max<int64_t>(elem, 16);

  // ---- single-mode fast path: per-system term programs ---------------------------------
  if (nm == 1) {
    size_t m1_max = 0;
    int max_side = 0;
    bool ok = true;
    std::vector<bq::M1Sys> progs;
    for (int b = 0; b < B && ok; ++b) {
      const Compiled& C = P.comp[b];
      bq::M1Sys m;
      std::memset(&m, 0, sizeof(m));
      const int M = C.M[0];
      if (C.r_diag) { ok = false; break; }  // diagonal residual layout: tiled kernel only
      m.M = M; m.has_sep = C.has_sep; m.has_r = C.has_r;
      for (int t = 0; t < (int)C.terms.size() && ok; ++t) {
        const TermDesc& td = C.terms[t];
        if (td.diagp1 && td.side != bq::SIDE_S) { ok = false; break; }
        const int woff = P.wbase[b];
        if (td.side == bq::SIDE_X) {
          if (m.nX == BQ_M1_MAXT) { ok = false; break; }
          m.sX[m.nX] = td.deltaGx; m.wX[m.nX] = td.n_act ? td.wtab[0] + woff : -1; m.tX[m.nX++] = t;
        } else if (td.side == bq::SIDE_Y) {
          if (m.nY == BQ_M1_MAXT) { ok = false; break; }
          m.sY[m.nY] = td.deltaGy; m.wY[m.nY] = td.n_act ? td.wtab[0] + woff : -1; m.tY[m.nY++] = t;
        } else {
          if (m.nS == BQ_M1_MAXT) { ok = false; break; }
          if (td.diagp1) m.sdiag |= 1 << m.nS;  // single mode: only where k = l
          m.sSx[m.nS] = td.deltaGx; m.sSy[m.nS] = td.deltaGy; m.wSx[m.nS] = -1; m.wSy[m.nS] = -1;
          for (int a = 0; a < td.n_act; ++a) {
            if (td.dim[a] == 0) m.wSx[m.nS] = td.wtab[a] + woff; else m.wSy[m.nS] = td.wtab[a] + woff;
          }
          m.tS[m.nS++] = t;
        }
      }
      max_side = std::max(max_side, std::max(m.nX, std::max(m.nY, m.nS)));
      const size_t bytes = (size_t)((C.has_r ? M * M : 0) + 4 * M) * cs + (size_t)(m.nX + m.nY + 2 * m.nS) * M * rs;
      if (bytes > 160 * 1024) ok = false;
      m1_max = std::max(m1_max, bytes);
      progs.push_back(m);
    }
    if (ok) {
      P.use_m1 = 1;
      P.m1_variant = max_side <= 2 ? 0 : 1;
      for (int i = 0; i < (int)P.sys.size(); ++i) {
        const SysDesc& sd = P.sys[i];
        bq::M1Sys m = progs[sd.prob];
        m.term_off = sd.term_off; m.diag_off = sd.diag_off;
        m.off_gx = sd.off_gx; m.off_gy = sd.off_gy; m.off_r = sd.off_r;
        m.c_re = sd.c_re; m.c_im = sd.c_im;
        P.m1.push_back(m);
        WorkItem w{i, 0, sd.has_r ? sd.n_r : 0, 0, sd.has_sep ? 2 * sd.n_g : 0, 0, sd.has_r ? sd.n_r : 0, 0, 0};
        P.work.push_back(w);
      }
      P.smem_bytes = (int)m1_max;
      // batched persistent solve: systems up to 1792 points, at most 2 terms per side
      bool solve_ok = P.m1_variant == 0;
      size_t solve_max = 0;
      std::vector<std::pair<int, int>> sz;
      for (int i = 0; i < (int)P.m1.size() && solve_ok; ++i) {
        const bq::M1Sys& m = P.m1[i];
        const int ntot = (m.has_r ? m.M * m.M : 0) + (m.has_sep ? 2 * m.M : 0);
        if (ntot > 1792) solve_ok = false;
        const size_t bytes = (size_t)(2 * ntot + 2 * m.M) * cs + (size_t)(m.nX + m.nY + 2 * m.nS) * m.M * rs;
        solve_max = std::max(solve_max, bytes);
        sz.push_back({-ntot, i});
      }
      // pipelined stage kernel: parameter blocks per problem, records per system
      {
        std::vector<int> poff(B, -1), pbytes(B, 0), pmerged(B, 0), pch0(B, -1), pch1(B, -1);
        std::vector<int> pgauss(B, 0);   // the problem's only envelope is a Gaussian (FP32 records)
        std::vector<float> pgpar(5 * (size_t)B, 0.f);
        size_t blk_max = 0, par_max = 0;
        bool pipe_ok = P.total_elems < ((int64_t)1 << 31);  // 32-bit element offsets
        int mmax = 1;
        std::vector<int> prob_terms(B, 0);  // offset of every problem's terms in P.terms (global channel indices)
        for (const SysDesc& sd : P.sys) prob_terms[sd.prob] = sd.term_off;
        for (int b = 0; b < B; ++b) {
          const Compiled& C = P.comp[b];
          const bq::M1Sys& m = progs[b];
          const int M = C.M[0];
          mmax = std::max(mmax, M);
          bq::PipeHdr hd;
          std::memset(&hd, 0, sizeof(hd));
          hd.M = M; hd.nX = m.nX; hd.nY = m.nY; hd.nS = m.nS; hd.has_sep = C.has_sep; hd.has_r = C.has_r;
          hd.sdiag = m.sdiag;
          hd.ntot = (C.has_r ? M * M : 0) + (C.has_sep ? 2 * M : 0);
          hd.n_terms = m.nX + m.nY + m.nS;
          for (int q = 0; q < BQ_M1_MAXT; ++q) { hd.sX[q] = m.sX[q]; hd.sY[q] = m.sY[q]; hd.sSx[q] = m.sSx[q]; hd.sSy[q] = m.sSy[q]; }
          {
            bool mg = M <= BQ_MERGED_MAXM && m.nS <= 2 && (P.m1_variant == 0 || m.nS <= 2);
            for (int q = 0; q < m.nX; ++q) mg = mg && std::abs(m.sX[q]) <= 1;
            for (int q = 0; q < m.nY; ++q) mg = mg && std::abs(m.sY[q]) <= 1;
            for (int q = 0; q < m.nS; ++q) mg = mg && std::abs(m.sSx[q]) <= 1 && std::abs(m.sSy[q]) <= 1;
            // the merged path stores MS = 2 (variant 0) or BQ_M1_MAXT (variant 1) sandwich records
            hd.merged = mg ? 1 : 0;
            pmerged[b] = hd.merged;
          }
          std::vector<unsigned char> blk(sizeof(hd));
          std::memcpy(blk.data(), &hd, sizeof(hd));
          auto put_c = [&](cplx v) {
            if (cs == 16) { double d[2] = {v.real(), v.imag()}; blk.insert(blk.end(), (unsigned char*)d, (unsigned char*)d + 16); }
            else { float f[2] = {(float)v.real(), (float)v.imag()}; blk.insert(blk.end(), (unsigned char*)f, (unsigned char*)f + 8); }
          };
          auto put_r = [&](double v) {
            if (rs == 8) blk.insert(blk.end(), (unsigned char*)&v, (unsigned char*)&v + 8);
            else { float f = (float)v; blk.insert(blk.end(), (unsigned char*)&f, (unsigned char*)&f + 4); }
          };
          // stage coefficients of the X, Y, S terms in program order: static part, and the
          // record's channel slot (at most two distinct channels per problem on this path)
          for (int q = 0; q < hd.n_terms; ++q) {
            const int t = q < m.nX ? m.tX[q] : (q < m.nX + m.nY ? m.tY[q - m.nX] : m.tS[q - m.nX - m.nY]);
            const TermDesc& td = P.terms[prob_terms[b] + t];
            int slot = -1;
            if (td.ch >= 0) {
              if (pch0[b] < 0 || pch0[b] == td.ch) { pch0[b] = td.ch; slot = 0; }
              else if (pch1[b] < 0 || pch1[b] == td.ch) { pch1[b] = td.ch; slot = 1; }
              else pipe_ok = false;
            }
            const size_t rec0 = blk.size();
            put_c(cplx(td.c_re, td.c_im));
            const int ci[2] = {slot, td.conj ? 1 : 0};
            blk.insert(blk.end(), (const unsigned char*)ci, (const unsigned char*)ci + 8);
            while (blk.size() - rec0 < sizeof(bq::PipeCoef<double2>) && cs == 16) blk.push_back(0);
          }
          // the envelopes themselves, so that the kernel evaluates them from the block
          const int chs[2] = {pch0[b], pch1[b]};
          int n_ch = 0;
          for (int c = 0; c < 2; ++c) {
            if (chs[c] < 0) break;
            const ChanDesc& cd = P.chans[chs[c]];
            bq::PipeChan pc;
            std::memset(&pc, 0, sizeof(pc));
            for (int i = 0; i < 4 && i < cd.n_par; ++i) pc.p[i] = P.chpar[cd.par_off + i];
            pc.f[0] = (float)pc.p[0];
            pc.f[1] = (float)pc.p[1];
            pc.f[2] = cd.kind == BQ_CH_GAUSS ? (float)(1.0 / (2.0 * pc.p[3] * pc.p[3])) : 0.f;
            pc.f[3] = cd.kind == BQ_CH_GAUSS ? (float)pc.p[2] : 0.f;
            pc.c_lo = cd.kind == BQ_CH_GAUSS ? (float)(pc.p[2] - (double)pc.f[3]) : 0.f;
            pc.kind = cd.kind;
            pc.par_off = cd.par_off;
            pc.n_par = cd.n_par;
            blk.insert(blk.end(), (const unsigned char*)&pc, (const unsigned char*)&pc + sizeof(pc));
            ++n_ch;
          }
          reinterpret_cast<bq::PipeHdr*>(blk.data())->n_ch = n_ch;
          if (n_ch == 1 && P.chans[chs[0]].kind == BQ_CH_GAUSS) {
            // the same FP32 values as the block's record (pc.f, pc.c_lo above)
            const double* cp = P.chpar.data() + P.chans[chs[0]].par_off;
            float* g = pgpar.data() + 5 * (size_t)b;
            g[0] = (float)cp[0];
            g[1] = (float)cp[1];
            g[2] = (float)(1.0 / (2.0 * cp[3] * cp[3]));
            g[3] = (float)cp[2];
            g[4] = (float)(cp[2] - (double)g[3]);
            pgauss[b] = 1;
          }
          for (int i = 0; i < M; ++i) put_c(C.diag[i]);
          for (int i = 0; i < M; ++i) put_c(C.diag[M + i]);
          auto put_w = [&](int woff) { for (int i = 0; i < M; ++i) put_r(woff >= 0 ? C.wtab[woff + i] : 1.0); };
          auto local = [&](int w) { return w >= 0 ? w - P.wbase[b] : -1; };
          for (int q = 0; q < m.nX; ++q) put_w(local(m.wX[q] >= 0 ? m.wX[q] : -1) >= 0 ? local(m.wX[q]) : -1);
          for (int q = 0; q < m.nY; ++q) put_w(m.wY[q] >= 0 ? local(m.wY[q]) : -1);
          for (int q = 0; q < m.nS; ++q) put_w(m.wSx[q] >= 0 ? local(m.wSx[q]) : -1);
          for (int q = 0; q < m.nS; ++q) put_w(m.wSy[q] >= 0 ? local(m.wSy[q]) : -1);
          while (blk.size() % 16) blk.push_back(0);
          // the problem's Tr(rho0 A) entries, one per lane of the warp that evaluates the
          // observable in the last stage (a larger support leaves it to the evaluation kernel)
          {
            const EvalGroup& g = P.groups[b];
            auto* hp = reinterpret_cast<bq::PipeHdr*>(blk.data());
            hp->obs_off = (int)blk.size();
            hp->n_obs = g.n_e <= 32 ? g.n_e : 0;
            if (g.n_e > 32) P.pipe_obs = 0;
            for (int e = 0; e < hp->n_obs; ++e) {
              const EvalEntry& en = P.entries[g.e_off + e];
              if (cs == 16) {
                bq::PipeObs<double2> o;
                std::memset(&o, 0, sizeof(o));
                o.kx = en.kx; o.ly = en.ly; o.f = make_double2(en.f_re, en.f_im);
                blk.insert(blk.end(), (const unsigned char*)&o, (const unsigned char*)&o + sizeof(o));
              } else {
                bq::PipeObs<float2> o;
                o.kx = en.kx; o.ly = en.ly; o.f = make_float2((float)en.f_re, (float)en.f_im);
                blk.insert(blk.end(), (const unsigned char*)&o, (const unsigned char*)&o + sizeof(o));
              }
            }
          }
          while (blk.size() % 16) blk.push_back(0);
          poff[b] = (int)P.pparams.size();
          pbytes[b] = (int)blk.size();
          P.pparams.insert(P.pparams.end(), blk.begin(), blk.end());
          par_max = std::max(par_max, blk.size());
        }
        static_assert(sizeof(bq::PipeCoef<float2>) == 16 && sizeof(bq::PipeCoef<double2>) == 32,
                      "coefficient records as written above");
        static_assert(sizeof(bq::PipeObs<float2>) == 16 && sizeof(bq::PipeObs<double2>) == 32,
                      "entry records keep the block 16-B aligned");
        static_assert(sizeof(bq::PipeRec) == 96, "two batches of records in the kernel's static shared memory");
        for (int i = 0; i < (int)P.sys.size(); ++i) {
          const SysDesc& sd = P.sys[i];
          bq::PipeRec r;
          std::memset(&r, 0, sizeof(r));
          const int pg = (int)(sd.has_sep ? sd.off_gy - sd.off_gx : 0);  // padded G_x length
          const int pr = (sd.n_r + 3) & ~3;
          r.blk_off = (int)(sd.has_sep ? sd.off_gx : sd.off_r);
          r.blk_elems = (sd.has_sep ? 2 * pg : 0) + (sd.has_r ? pr : 0);
          r.param_off = poff[sd.prob];
          r.param_bytes = pbytes[sd.prob];
          r.gy_off = sd.has_sep ? pg : -1;
          r.r_off = sd.has_r ? (sd.has_sep ? 2 * pg : 0) : -1;
          r.M = P.comp[sd.prob].M[0];
          r.merged = pmerged[sd.prob];
          r.nb = std::max(1, std::min(BQ_PIPE_THREADS / r.M, r.M));
          r.rb = (r.M + r.nb - 1) / r.nb;
          r.inv_m = 1.0f / (float)r.M;
          if (cs == 16) {
            r.d.c_re = sd.c_re;
            r.d.c_im = sd.c_im;
            r.d.w_re = sd.w_re;
            r.d.w_im = sd.w_im;
          } else if (pgauss[sd.prob]) {
            const float* g = pgpar.data() + 5 * (size_t)sd.prob;
            r.f.amp_re = g[0];
            r.f.amp_im = g[1];
            r.f.k = g[2];
            r.f.c_hi = g[3];
            r.f.c_lo = g[4];
            r.f.gauss = 1;
          }
          r.w32_re = (float)sd.w_re;
          r.w32_im = (float)sd.w_im;
          r.c32_re = (float)sd.c_re;
          r.c32_im = (float)sd.c_im;
          r.sys = i;
          P.precs.push_back(r);
          blk_max = std::max(blk_max, (size_t)r.blk_elems);
        }
        // Within each run of kPipeSortRun consecutive systems, largest first: CTA b takes
        // records b, b + G, b + 2G, ..., so every CTA gets one system of each size band of a
        // run and the CTAs finish together (in problem order a CTA's load is a sum of a few
        // random sizes, and the slowest CTA sets the stage's time).  Sorting only within runs
        // keeps the systems in flight at any moment in one region of the state arrays.
        const size_t kPipeSortRun = 4096;
        for (size_t r0 = 0; r0 < P.precs.size(); r0 += kPipeSortRun)
          std::stable_sort(P.precs.begin() + r0, P.precs.begin() + std::min(P.precs.size(), r0 + kPipeSortRun),
                           [](const bq::PipeRec& a, const bq::PipeRec& b) { return a.blk_elems > b.blk_elems; });
        // Shared-memory slot: [parameter block | guard | stage input | guard].  Neighbour reads
        // at a system's edges reach at most M + 1 elements before or after its block (the
        // sandwich source (k - 1, l - 1) at k = 0 of a block without G), so each guard holds
        // mmax + 2 elements, rounded to 4.
        auto a128 = [](size_t x) { return (x + 127) & ~(size_t)127; };
        const size_t guard = (size_t)((mmax + 2 + 3) & ~3);
        const size_t zero0 = a128(par_max);
        P.pipe_zero_off = (int)zero0;
        P.pipe_off_u = (int)(zero0 + guard * cs);
        P.pipe_zero_bytes = (int)((2 * guard + blk_max) * cs);
        P.pipe_slot = (int)a128(zero0 + P.pipe_zero_bytes);
        P.pipe_mmax = mmax;
        P.use_pipe = pipe_ok && 2 * (size_t)P.pipe_slot <= 200 * 1024 ? 1 : 0;

      }
      if (solve_ok && solve_max <= 160 * 1024) {
        std::stable_sort(sz.begin(), sz.end());
        for (auto& e : sz) P.order.push_back(e.second);
        P.solve_smem = (int)solve_max;
        // merged-stencil persistent solve: shifts in {-1, 0, 1}, <= 2 sandwich terms,
        // column strips of an even number of rows, at most 8, with 256 threads (M <= 42)
        bool mg = true;
        size_t mg_max = 0;
        for (int i = 0; i < (int)P.m1.size() && mg; ++i) {
          const bq::M1Sys& m = P.m1[i];
          const int M = m.M;
          const int np = (M + 1) / 2;  // strips of an even number of rows (k_solve_mg)
          const int nb = std::min(256 / M, np);
          mg = mg && M >= 1 && nb >= 1 && 2 * ((np + nb - 1) / nb) <= 8 && m.nS <= 2;
          for (int q = 0; q < m.nX; ++q) mg = mg && std::abs(m.sX[q]) <= 1;
          for (int q = 0; q < m.nY; ++q) mg = mg && std::abs(m.sY[q]) <= 1;
          for (int q = 0; q < m.nS; ++q) mg = mg && std::abs(m.sSx[q]) <= 1 && std::abs(m.sSy[q]) <= 1;
          const int ntot = (m.has_r ? M * M : 0) + (m.has_sep ? 2 * M : 0);
          const int nr = m.has_r ? M * M : 0;  // stage sum and compensation of the R points
          mg_max = std::max(mg_max, (size_t)(2 * ntot + 2 * nr + 2 * M + 2 * 8 * M) * cs +
                                        (size_t)(m.nX + m.nY + 2 * m.nS) * M * rs);
        }
        if (mg && mg_max <= 160 * 1024) { P.solve_mg = 1; P.solve_mg_smem = (int)mg_max; }
      }
    }
  }

  // ---- work items (tiles of R; the first tile of a system also updates G_x, G_y) ------
  for (SysDesc& sd : P.sys) {
    int ns = 0, cw = 0;
    for (auto& td : P.comp[sd.prob].terms) {
      ns += td.side == bq::SIDE_S;
      cw += td.n_act > 0 ? sd.M[td.dim[0] % sd.nm] : 1;
    }
    sd.n_sterms = ns;
    sd.cw_elems = cw;
    P.srcred_stride = std::max(P.srcred_stride, (sd.has_sep && sd.has_r) ? 2 * ns * sd.n_g : 0);
    P.max_s = std::max(P.max_s, (sd.has_sep && sd.has_r) ? ns : 0);
  }
  if (!P.use_m1) {
    int smem_max = 0, adj_max = 0;
    build_work(P.sys, cs, 0, 0, P.work, smem_max, adj_max);
    P.smem_bytes = (int)(smem_max * cs);
    P.adj_smem = (int)(adj_max * cs);
    // capacity for the smallest tile the schedules may choose
    std::vector<WorkItem> wmin;
    int smin = 0, amin = 0;
    build_work(P.sys, cs, 32, 0, wmin, smin, amin);
    P.work_cap = std::max(P.work.size(), wmin.size());
  } else {  // one-CTA-per-system items (whole system as the window) for the adjoint kernel
    size_t adj_max = 0;
    for (auto& w : P.work) {
      const SysDesc& sd = P.sys[w.sys];
      adj_max = std::max(adj_max, (size_t)(w.win_hi - w.win_lo) +
                                      (sd.has_sep ? (size_t)(2 + 2 * sd.n_sterms) * sd.n_g : 0));
    }
    P.adj_smem = (int)(adj_max * cs);
  }
  P.dt_max = 2.0 * std::sqrt(2.0) / std::max(P.rho, 1e-300);
  if (o->dt > 0.0 && o->dt > P.dt_max)
    return fail(BQ_EUNSTABLE_DT, "dt=%g above the RK4 stability bound %g (spectral bound %g)", o->dt, P.dt_max, P.rho);

  // ---- layout -------------------------------------------------------------------------
  Layout& L = P.L;
  size_t o2 = 0;
  auto seg = [&](size_t bytes) { size_t s = o2; o2 = align_up(o2 + std::max<size_t>(bytes, 1)); return s; };
  L.off_sys = seg(P.sys.size() * sizeof(SysDesc));
  L.off_terms = seg(P.terms.size() * sizeof(TermDesc));
  L.off_chans = seg(P.chans.size() * sizeof(ChanDesc));
  L.off_chpar = seg(P.chpar.size() * sizeof(double));
  L.off_work = seg(std::max(P.work.size(), P.work_cap) * sizeof(WorkItem));
  L.off_m1 = seg(P.m1.size() * sizeof(bq::M1Sys));
  L.off_order = seg(P.order.size() * sizeof(int));
  L.off_pparams = seg(P.pparams.size());
  L.off_precs = seg(P.precs.size() * sizeof(bq::PipeRec));
  L.off_obs = seg(P.use_pipe ? P.sys.size() * sizeof(double2) : 0);
  L.off_dc = seg(P.dc.size() * sizeof(double2));
  L.off_groups = seg(P.groups.size() * sizeof(EvalGroup));
  L.off_entries = seg(P.entries.size() * sizeof(EvalEntry));
  L.off_out = seg(P.groups.size() * 2 * sizeof(double));
  L.off_wtab = seg(P.wtab.size() * rs);
  L.off_diag = seg(P.diag.size() * cs);
  L.off_ctrl = seg(64);
  L.off_init = seg(P.init.size() * sizeof(InitEntry));
  const size_t sbytes = (size_t)P.total_elems * cs;
  L.off_y = seg(sbytes);
  L.off_comp = seg(sbytes);
  L.off_ua = seg(sbytes);
  L.off_ub = seg(sbytes);
  L.off_acc = seg(sbytes);
  L.total = o2;
  return BQ_OK;
}

// Slots and grid of the pipelined stage kernel for `slots` shared-memory slots per CTA and
// at most `cap` resident CTAs per SM (0: the occupancy limit).  BQ_EUNSUPPORTED when the
// slots do not fit.
static int pipe_configure(bq_state* st, int slots, int cap) {
  if (slots < 2 || slots > 4) return fail(BQ_EUNSUPPORTED, "pipe_slots must be 2..4");
  int dev = 0, nsm = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  int grid[4];
  for (int q = 0; q < 4; ++q) {  // one kernel per RK4 stage
    const size_t smem = (size_t)slots * st->pipe_slot[q] + st->pipe_mv_bytes;
    if (smem > BQ_MAX_DYN_SMEM) return fail(BQ_EUNSUPPORTED, "%d slots need %zu bytes of shared memory", slots, smem);
    int per_sm = 0;
    CUDA_TRY(bq::pipe_blocks_per_sm(st->dtype, st->m1_variant, q + 1, (int)smem, &per_sm));
    if (per_sm < 1) return fail(BQ_EUNSUPPORTED, "%d slots do not fit on an SM", slots);
    if (cap > 0) per_sm = std::min(per_sm, cap);
    grid[q] = std::min(st->n_sys, per_sm * nsm);
  }
  // the multi-step kernel holds all four stages: its own occupancy
  int per_sm = 0;
  CUDA_TRY(bq::steps_pipe_blocks_per_sm(st->dtype, st->m1_variant,
                                        (int)((size_t)slots * st->pipe_slot[0] + st->pipe_mv_bytes), &per_sm));
  if (cap > 0) per_sm = std::min(per_sm, cap);
  for (int q = 0; q < 4; ++q) { st->pipe_nslots[q] = slots; st->pipe_grid[q] = grid[q]; }
  st->pipe_steps_grid = per_sm > 0 ? std::min(st->n_sys, per_sm * nsm) : 0;
  st->pipe_cap = cap;
  return BQ_OK;
}

extern "C" int bq_required_bytes(const bq_problem* const* probs, int B, const bq_map_opts* opts, size_t* out) {
  if (!out) return fail(BQ_EINVAL, "out is NULL");
  Plan P;
  int r = make_plan(probs, B, opts, P);
  if (r != BQ_OK) return r;
  *out = P.L.total;
  return BQ_OK;
}

extern "C" int bq_plan(const bq_problem* const* probs, int B, const bq_map_opts* opts, bq_plan_info* out) {
  if (!out) return fail(BQ_EINVAL, "out is NULL");
  Plan P;
  int r = make_plan(probs, B, opts, P);
  if (r != BQ_OK) return r;
  std::memset(out, 0, sizeof(*out));
  out->n_systems = (int)P.sys.size();
  out->n_work = (int)P.work.size();
  out->work_cap = (int)std::max(P.work.size(), P.work_cap);
  out->lanes = default_lanes(P.sys);
  out->stage_variant = P.use_pipe ? 2 : (P.use_m1 ? 1 : 0);
  out->smem_bytes = P.smem_bytes;
  out->adj_smem_bytes = P.adj_smem;
  out->total_elems = P.total_elems;
  return BQ_OK;
}

template <typename T>
static std::vector<T> to_real(const std::vector<double>& v) { return std::vector<T>(v.begin(), v.end()); }

extern "C" int bq_map(const bq_problem* const* probs, int B, const bq_map_opts* o, void* pool, size_t pool_bytes,
                      void* stream, bq_state** out) {
  if (!out) return fail(BQ_EINVAL, "out is NULL");
  *out = nullptr;
  Plan P;
  int r = make_plan(probs, B, o, P);
  if (r != BQ_OK) return r;
  if (!pool || ((uintptr_t)pool & 255)) return fail(BQ_EINVAL, "device pool must be non-NULL and 256-byte aligned");
  if (pool_bytes < P.L.total) return fail(BQ_ENOMEM, "pool has %zu bytes, needs %zu", pool_bytes, P.L.total);
  const double dt_max = P.dt_max;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)pool;
  const Layout& L = P.L;
  auto up = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
    if (!bytes) return cudaSuccess;
    return cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, s);
  };
  CUDA_TRY(up(L.off_sys, P.sys.data(), P.sys.size() * sizeof(SysDesc)));
  CUDA_TRY(up(L.off_terms, P.terms.data(), P.terms.size() * sizeof(TermDesc)));
  CUDA_TRY(up(L.off_chans, P.chans.data(), P.chans.size() * sizeof(ChanDesc)));
  CUDA_TRY(up(L.off_chpar, P.chpar.data(), P.chpar.size() * sizeof(double)));
  CUDA_TRY(up(L.off_work, P.work.data(), P.work.size() * sizeof(WorkItem)));
  CUDA_TRY(up(L.off_m1, P.m1.data(), P.m1.size() * sizeof(bq::M1Sys)));
  CUDA_TRY(up(L.off_order, P.order.data(), P.order.size() * sizeof(int)));
  CUDA_TRY(up(L.off_pparams, P.pparams.data(), P.pparams.size()));
  CUDA_TRY(up(L.off_precs, P.precs.data(), P.precs.size() * sizeof(bq::PipeRec)));
  {
    std::vector<double2> dcv(P.dc.size());
    for (size_t i = 0; i < dcv.size(); ++i) dcv[i] = make_double2(P.dc[i].real(), P.dc[i].imag());
    CUDA_TRY(up(L.off_dc, dcv.data(), dcv.size() * sizeof(double2)));
  }
  CUDA_TRY(up(L.off_groups, P.groups.data(), P.groups.size() * sizeof(EvalGroup)));
  CUDA_TRY(up(L.off_entries, P.entries.data(), P.entries.size() * sizeof(EvalEntry)));
  if (o->dtype == BQ_F64) {
    CUDA_TRY(up(L.off_wtab, P.wtab.data(), P.wtab.size() * sizeof(double)));
    std::vector<double2> d(P.diag.size());
    for (size_t i = 0; i < d.size(); ++i) d[i] = make_double2(P.diag[i].real(), P.diag[i].imag());
    CUDA_TRY(up(L.off_diag, d.data(), d.size() * sizeof(double2)));
  } else {
    auto w = to_real<float>(P.wtab);
    CUDA_TRY(up(L.off_wtab, w.data(), w.size() * sizeof(float)));
    std::vector<float2> d(P.diag.size());
    for (size_t i = 0; i < d.size(); ++i) d[i] = make_float2((float)P.diag[i].real(), (float)P.diag[i].imag());
    CUDA_TRY(up(L.off_diag, d.data(), d.size() * sizeof(float2)));
  }
  CUDA_TRY(cudaMemsetAsync(base + L.off_ctrl, 0, 64, s));
  CUDA_TRY(up(L.off_init, P.init.data(), P.init.size() * sizeof(InitEntry)));
  const size_t cs = o->dtype == BQ_F64 ? 16 : 8;
  // the state arrays; the stage scratch too, so that the padding between a system's blocks
  // (never written by the stage kernels, read at a system's edges with zero coefficients)
  // holds finite values in every buffer the stage kernels read
  for (size_t off : {L.off_y, L.off_comp, L.off_ua, L.off_ub, L.off_acc})
    CUDA_TRY(cudaMemsetAsync(base + off, 0, (size_t)P.total_elems * cs, s));
  CUDA_TRY(bq::launch_scatter((const InitEntry*)(base + L.off_init), (int)P.init.size(), base + L.off_y, o->dtype, s));
  g_launches++;
  CUDA_TRY(cudaStreamSynchronize(s));

  auto* st = new bq_state();
  st->B = B; st->nm = probs[0]->nm; st->dtype = o->dtype; st->method = o->method; st->basis = P.comp[0].basis;
  st->n_sys = (int)P.sys.size(); st->n_work = (int)P.work.size(); st->smem_bytes = P.smem_bytes;
  st->work_cap = (int)std::max(P.work.size(), P.work_cap);
  st->lanes = default_lanes(P.sys);
  st->use_m1 = P.use_m1;
  {
    int mt = 0, mb = 0;
    for (int g = 0; g < (int)P.groups.size(); ++g) {
      const int pairs = P.groups[g].n_sys * P.groups[g].n_e;
      if (g < P.n_trace_groups) mt = std::max(mt, pairs); else mb = std::max(mb, pairs);
    }
    st->trace_small = mt <= 8;
    st->block_small = mb <= 8;
  }
  st->m1_variant = P.m1_variant;
  st->solve_ok = P.order.empty() ? 0 : 1;
  st->use_pipe = P.use_pipe;
  for (const TermDesc& td : P.terms) st->has_diag = st->has_diag || td.diagp1 != 0;
  for (const SysDesc& sd : P.sys) st->r_diag = st->r_diag || sd.r_diag;
  for (const WorkItem& w : P.work) st->has_gread = st->has_gread || w.gread;
  st->pipe_off_u = P.pipe_off_u; st->pipe_zero_off = P.pipe_zero_off; st->pipe_zero_bytes = P.pipe_zero_bytes;
  st->pipe_mmax = P.pipe_mmax;
  st->pipe_obs = P.pipe_obs;
  for (int q = 0; q < 4; ++q) st->pipe_slot[q] = P.pipe_slot;
  {
    // row and column coefficient records of the merged path
    const int ms = P.m1_variant == 0 ? 2 : BQ_M1_MAXT;
    st->pipe_mv_bytes = (int)(((size_t)2 * BQ_PIPE_RS(ms) * BQ_MERGED_MAXM * (o->dtype == BQ_F64 ? 16 : 8) + 127) & ~(size_t)127);
  }
  if (st->use_pipe) {
    // double buffering at the occupancy limit; bq_autotune may pick another schedule
    int rc = pipe_configure(st, 2, 0);
    if (rc == BQ_ECUDA) return rc;
    st->use_pipe = rc == BQ_OK ? 1 : 0;
  }
  st->pipe_ok = st->use_pipe;

  st->grad_size = P.grad_size;
  st->adj_smem = P.adj_smem;
  st->srcred_stride = P.srcred_stride;
  for (const SysDesc& sd : P.sys) st->ng_max = std::max(st->ng_max, sd.n_g);
  st->max_s = P.max_s;
  st->terms_host = P.terms;
  st->chans_host = P.chans;
  st->chpar_host = P.chpar;
  st->solve_smem = P.solve_smem;
  st->solve_mg = P.solve_mg;
  st->solve_mg_ok = P.solve_mg;
  st->solve_mg_smem = P.solve_mg_smem;
  st->n_trace_groups = P.n_trace_groups; st->n_block_groups = P.n_block_groups; st->block_dim = P.block_dim;
  st->total_elems = P.total_elems; st->dt_max = dt_max; st->horizon = o->horizon; st->reverse = o->reverse_time;
  st->pool = base; st->L = L; st->sys = P.sys;
  for (int b = 0; b < B; ++b) for (int j = 0; j < BQ_MAX_MODES; ++j) st->prob_M.push_back(P.comp[b].M[j]);
  *out = st;
  return BQ_OK;
}

extern "C" void bq_state_destroy(bq_state* s) {
  if (!s) return;
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  for (cudaStream_t& gs : s->grad_stream)
    if (gs) cudaStreamDestroy(gs);
  delete s;
}

// ---------------------------------------------------------------------------------------
// Stepping.
// ---------------------------------------------------------------------------------------
static bq::StageArgs stage_args(bq_state* s, int stage, double dt) {
  bq::StageArgs a;
  std::memset(&a, 0, sizeof(a));  // every field, including the optional recording pointer
  char* b = s->pool;
  const Layout& L = s->L;
  a.sys = (const SysDesc*)(b + L.off_sys);
  a.terms = (const TermDesc*)(b + L.off_terms);
  a.chans = (const ChanDesc*)(b + L.off_chans);
  a.chpar = (const double*)(b + L.off_chpar);
  a.wtab = b + L.off_wtab;
  a.diag = b + L.off_diag;
  a.work = (const WorkItem*)(b + L.off_work);
  // ping-pong: stage 1 reads y -> ua; 2 reads ua -> ub; 3 reads ub -> ua; 4 reads ua -> y
  void* y = b + L.off_y;
  void* ua = b + L.off_ua;
  void* ub = b + L.off_ub;
  a.u_in = stage == 1 ? y : (stage == 2 ? ua : (stage == 3 ? ub : ua));
  a.u_out = stage == 1 ? ua : (stage == 2 ? ub : (stage == 3 ? ua : nullptr));
  a.y = y;
  a.acc = b + L.off_acc;
  a.comp = b + L.off_comp;
  a.tau_base = (const double*)(b + L.off_ctrl);
  a.counter = (long long*)(b + L.off_ctrl + 8);
  a.ticket = (unsigned int*)(b + L.off_ctrl + 16);
  a.dt = dt;
  a.horizon = s->horizon;
  a.reverse = s->reverse;
  a.stage = stage;
  a.lanes = s->lanes;
  return a;
}

// kernels enqueued by one stage launch (the pipelined kernel evaluates its drive envelopes itself)
static int kernels_per_stage(const bq_state*, bool) { return 1; }

// bq_step's pipelined path runs the four stages of a step in one kernel (k_steps_pipe)
static bool pipe_fused_on(const bq_state* s) { return s->use_pipe && s->pipe_fused && s->pipe_steps_grid > 0; }
// kernels bq_step enqueues per RK4 step
static int kernels_per_step(const bq_state* s) { return pipe_fused_on(s) ? 1 : 4 * kernels_per_stage(s, false); }

// comp holds the rounding residual of the last state update (true state = y - comp).  After
// bq_load_state it is zero by definition but not written yet: the pipelined kernel skips
// reading it at its next stage 1, and every other consumer of the raw arrays clears it first
// (asynchronous on st).
static cudaError_t ensure_comp(bq_state* s, cudaStream_t st) {
  if (!s->comp_zero) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(s->pool + s->L.off_comp, 0, (size_t)s->total_elems * (s->dtype == BQ_F64 ? 16 : 8), st);
  if (e != cudaSuccess) return e;
  s->comp_zero = 0;
  return cudaSuccess;
}

// Arguments of the pipelined kernels for stage a.stage (1..4) of a.
static bq::PipeArgs pipe_args(bq_state* s, const bq::StageArgs& a) {
  char* b = s->pool;
  const Layout& L = s->L;
  bq::PipeArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.recs = (const bq::PipeRec*)(b + L.off_precs);
  pa.params = (const unsigned char*)(b + L.off_pparams);
  pa.chans = a.chans;
  pa.chpar = a.chpar;
  pa.u_in = a.u_in; pa.u_out = a.u_out; pa.y = a.y; pa.acc = a.acc; pa.comp = a.comp;
  pa.ticket = a.ticket; pa.counter = a.counter; pa.tau_base = a.tau_base;
  pa.error = (unsigned int*)(b + L.off_ctrl + 32);
  pa.n_sys = s->n_sys;
  const int q = a.stage - 1;
  pa.n_slots = s->pipe_nslots[q];
  pa.slot_bytes = s->pipe_slot[q];
  pa.off_u = s->pipe_off_u;
  pa.zero_off = s->pipe_zero_off;
  pa.zero_bytes = s->pipe_zero_bytes;
  pa.mmax = s->pipe_mmax;
  pa.reverse = a.reverse;
  pa.comp_zero = a.stage == 1 ? s->comp_zero : 0;
  pa.obs = s->pipe_obs ? (double2*)(b + L.off_obs) : nullptr;
  pa.dt = a.dt;
  pa.horizon = a.horizon;
  return pa;
}

static cudaError_t launch_any_stage(bq_state* s, const bq::StageArgs& a, cudaStream_t st) {
  if (s->use_pipe && !a.rec) {
    const bq::PipeArgs pa = pipe_args(s, a);
    const int q = a.stage - 1;
    s->obs_valid = a.stage == 4 && s->pipe_obs;
    if (a.stage == 1) s->comp_zero = 0;  // stage 4 of this step writes comp everywhere
    return bq::launch_stage_pipe(pa, s->m1_variant, s->dtype, a.stage, s->pipe_grid[q],
                                 pa.n_slots * pa.slot_bytes + s->pipe_mv_bytes, st);
  }
  s->obs_valid = 0;
  if (s->use_m1)
    return bq::launch_stage_m1(a, (const bq::M1Sys*)(s->pool + s->L.off_m1), s->m1_variant, s->dtype, s->n_work,
                               s->smem_bytes, st);
  return bq::launch_stage(a, s->dtype, s->nm, s->n_work, s->smem_bytes, st);
}

static cudaError_t enqueue_steps(bq_state* s, double dt, int64_t n, cudaStream_t st) {
  if (pipe_fused_on(s)) {
    // The four stages of a step in one launch of the multi-step kernel, one launch per step.
    // (Several steps per launch were slower, 146 against 110 us per step on a 4096-system
    // batch whose arrays fit in L2 and 1.95 against 1.43 ms on 65 536 systems: without the
    // launch boundary the CTAs drift apart by stages and the data in flight outgrows L2 and
    // spreads over the arrays in HBM.)
    for (int64_t i = 0; i < n; ++i) {
      const bq::PipeArgs pa = pipe_args(s, stage_args(s, 1, dt));
      s->comp_zero = 0;
      s->obs_valid = s->pipe_obs;
      cudaError_t e = bq::launch_steps_pipe(pa, s->pool + s->L.off_ua, s->pool + s->L.off_ub, 1, s->m1_variant,
                                            s->dtype, s->pipe_steps_grid,
                                            pa.n_slots * pa.slot_bytes + s->pipe_mv_bytes, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int stage = 1; stage <= 4; ++stage) {
      cudaError_t e = launch_any_stage(s, stage_args(s, stage, dt), st);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

static const int kGraphSteps = 64;

extern "C" int bq_step(bq_state* s, double dt, int64_t n_steps, void* stream) {
  if (!s) return fail(BQ_EINVAL, "state is NULL");
  if (n_steps < 0) return fail(BQ_EINVAL, "n_steps < 0");
  if (!(dt > 0.0)) return fail(BQ_EINVAL, "dt must be > 0");
  if (dt > s->dt_max * (1.0 + 1e-12))
    return fail(BQ_EUNSTABLE_DT, "dt=%g above the RK4 stability bound %g", dt, s->dt_max);
  if (n_steps == 0) return BQ_OK;
  cudaStream_t st = (cudaStream_t)stream;
  char* b = s->pool;
  if (!s->use_pipe) CUDA_TRY(ensure_comp(s, st));
  // tau at the start of this call; the stage kernels add counter * dt
  s->tau_base_host = s->tau;
  CUDA_TRY(cudaMemcpyAsync(b + s->L.off_ctrl, &s->tau_base_host, sizeof(double), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemsetAsync(b + s->L.off_ctrl + 8, 0, 16, st));
  int64_t left = n_steps;
  if (n_steps >= kGraphSteps) {
    CUDA_TRY(ensure_comp(s, st));  // the graph must not carry a first stage that skips comp
    if (!s->graph || s->graph_dt != dt) {
      if (s->graph) { cudaGraphExecDestroy(s->graph); s->graph = nullptr; }
      if (!s->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
      cudaGraph_t g;
      CUDA_TRY(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = enqueue_steps(s, dt, kGraphSteps, s->cap_stream);
      cudaError_t e2 = cudaStreamEndCapture(s->cap_stream, &g);
      if (e != cudaSuccess) return fail(BQ_ECUDA, "capture: %s", cudaGetErrorString(e));
      if (e2 != cudaSuccess) return fail(BQ_ECUDA, "end capture: %s", cudaGetErrorString(e2));
      CUDA_TRY(cudaGraphInstantiate(&s->graph, g, 0));
      cudaGraphDestroy(g);
      s->graph_dt = dt;
    }
    while (left >= kGraphSteps) {
      CUDA_TRY(cudaGraphLaunch(s->graph, st));
      g_launches += kGraphSteps * kernels_per_step(s);
      left -= kGraphSteps;
    }
  }
  if (left > 0) {
    CUDA_TRY(enqueue_steps(s, dt, left, st));
    g_launches += left * kernels_per_step(s);
  }
  s->tau += (double)n_steps * dt;
  return BQ_OK;
}

// Same stepping as bq_step, with the RK4 scratch taken from the library's fixed device
// array (see bq_step_fixed_scratch in bq.h).  No allocation of any kind: plain launches,
// no CUDA graph.
extern "C" int bq_step_fixed_scratch(bq_state* s, double dt, int64_t n_steps, void* stream) {
  if (!s) return fail(BQ_EINVAL, "state is NULL");
  if (n_steps < 0) return fail(BQ_EINVAL, "n_steps < 0");
  if (!(dt > 0.0)) return fail(BQ_EINVAL, "dt must be > 0");
  if (dt > s->dt_max * (1.0 + 1e-12))
    return fail(BQ_EUNSTABLE_DT, "dt=%g above the RK4 stability bound %g", dt, s->dt_max);
  const size_t need = (size_t)s->total_elems * (s->dtype == BQ_F64 ? 16 : 8);
  if (need > BQ_FIXED_SCRATCH_BYTES)
    return fail(BQ_EUNSUPPORTED, "state needs %zu bytes per scratch buffer; the fixed scratch holds %u "
                "(use bq_step for larger states)", need, (unsigned)BQ_FIXED_SCRATCH_BYTES);
  if (n_steps == 0) return BQ_OK;
  void* scratch = nullptr;
  CUDA_TRY(bq::fixed_scratch(&scratch));
  char* ua = (char*)scratch;
  char* ub = ua + BQ_FIXED_SCRATCH_BYTES;
  char* acc = ub + BQ_FIXED_SCRATCH_BYTES;
  cudaStream_t st = (cudaStream_t)stream;
  char* b = s->pool;
  if (!s->use_pipe) CUDA_TRY(ensure_comp(s, st));
  // The array keeps whatever earlier calls (possibly of other states, layouts or precisions)
  // left in it.  The stage kernels write every element of this state's systems before reading
  // it, but read the padding between a system's arrays at its edges (with zero coefficients):
  // clear the buffers' used range so that the padding holds zeros, not stale bit patterns that
  // could read as non-finite values in this precision.
  const size_t used = (size_t)s->total_elems * (s->dtype == BQ_F64 ? 16 : 8);
  CUDA_TRY(cudaMemsetAsync(ua, 0, used, st));
  CUDA_TRY(cudaMemsetAsync(ub, 0, used, st));
  CUDA_TRY(cudaMemsetAsync(acc, 0, used, st));
  s->tau_base_host = s->tau;
  CUDA_TRY(cudaMemcpyAsync(b + s->L.off_ctrl, &s->tau_base_host, sizeof(double), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemsetAsync(b + s->L.off_ctrl + 8, 0, 16, st));
  for (int64_t i = 0; i < n_steps; ++i)
    for (int stage = 1; stage <= 4; ++stage) {
      bq::StageArgs a = stage_args(s, stage, dt);
      void* y = b + s->L.off_y;
      a.u_in = stage == 1 ? (const void*)y : (stage == 3 ? (const void*)ub : (const void*)ua);
      a.u_out = stage == 1 ? (void*)ua : (stage == 2 ? (void*)ub : (stage == 3 ? (void*)ua : nullptr));
      a.acc = acc;
      CUDA_TRY(launch_any_stage(s, a, st));
      g_launches += kernels_per_stage(s, false);
    }
  s->tau += (double)n_steps * dt;
  return BQ_OK;
}

static cudaError_t enqueue_solve(bq_state* s, double dt, int64_t n_steps, cudaStream_t st);

extern "C" int bq_solve(bq_state* s, double dt, int64_t n_steps, void* stream) {
  if (!s) return fail(BQ_EINVAL, "state is NULL");
  if (!s->solve_ok || s->solve_via_step) return bq_step(s, dt, n_steps, stream);
  if (n_steps < 0) return fail(BQ_EINVAL, "n_steps < 0");
  if (!(dt > 0.0)) return fail(BQ_EINVAL, "dt must be > 0");
  if (dt > s->dt_max * (1.0 + 1e-12))
    return fail(BQ_EUNSTABLE_DT, "dt=%g above the RK4 stability bound %g", dt, s->dt_max);
  if (n_steps == 0) return BQ_OK;
  CUDA_TRY(ensure_comp(s, (cudaStream_t)stream));
  CUDA_TRY(enqueue_solve(s, dt, n_steps, (cudaStream_t)stream));
  g_launches++;
  s->tau += (double)n_steps * dt;
  return BQ_OK;
}

// One persistent-solve launch of n_steps steps from s->tau with the state's schedule.
static cudaError_t enqueue_solve(bq_state* s, double dt, int64_t n_steps, cudaStream_t st) {
  char* b = s->pool;
  const Layout& L = s->L;
  s->obs_valid = 0;
  cudaError_t e = cudaMemsetAsync(b + L.off_ctrl + 24, 0, 8, st);
  if (e != cudaSuccess) return e;
  bq::SolveArgs a;
  std::memset(&a, 0, sizeof(a));
  a.m1 = (const bq::M1Sys*)(b + L.off_m1);
  a.order = (const int*)(b + L.off_order);
  a.terms = (const TermDesc*)(b + L.off_terms);
  a.chans = (const ChanDesc*)(b + L.off_chans);
  a.chpar = (const double*)(b + L.off_chpar);
  a.wtab = b + L.off_wtab;
  a.diag = b + L.off_diag;
  a.y = b + L.off_y;
  a.comp = b + L.off_comp;
  a.queue = (unsigned int*)(b + L.off_ctrl + 24);
  a.n_sys = s->n_sys;
  a.reverse = s->reverse;
  a.has_diag = s->has_diag;
  a.n_steps = n_steps;
  a.dt = dt;
  a.tau0 = s->tau;
  a.horizon = s->horizon;
  if (s->solve_mg) return bq::launch_solve_mg(a, s->dtype, s->solve_mg_smem, s->solve_cap, st, &s->last_solve_grid);
  return bq::launch_solve_m1(a, s->dtype, 0, s->solve_smem, s->solve_cap, st, &s->last_solve_grid);
}

extern "C" int bq_stage_variant(const bq_state* s, int* variant) {
  if (!s || !variant) return fail(BQ_EINVAL, "NULL argument");
  *variant = s->use_pipe ? 2 : (s->use_m1 ? 1 : 0);
  return BQ_OK;
}

extern "C" int bq_solve_eligible(const bq_state* s, int* eligible) {
  if (!s || !eligible) return fail(BQ_EINVAL, "NULL argument");
  *eligible = s->solve_ok;
  return BQ_OK;
}

// ---------------------------------------------------------------------------------------
// Schedules and the autotuner.
// ---------------------------------------------------------------------------------------
static void drop_graph(bq_state* s) {
  if (s->graph) { cudaGraphExecDestroy(s->graph); s->graph = nullptr; }
}

// Rewrites the tiled kernel's work items for tile length `tile` (0 = default) and global-read
// tiles on request.
static int apply_tile(bq_state* s, int tile, int gread) {
  if (s->use_m1) return fail(BQ_EUNSUPPORTED, "single-mode states have no tiled work items");
  if (tile != 0 && tile < 32) return fail(BQ_EINVAL, "tile must be 0 or >= 32");
  const size_t cs = s->dtype == BQ_F64 ? 16 : 8;
  std::vector<WorkItem> work;
  int smem = 0, adj = 0;
  build_work(s->sys, cs, tile, gread, work, smem, adj);
  if ((int)work.size() > s->work_cap) return fail(BQ_EUNSUPPORTED, "tile %d needs %zu work items > %d", tile, work.size(), s->work_cap);
  if ((size_t)smem * cs > BQ_MAX_DYN_SMEM || (size_t)adj * cs > BQ_MAX_DYN_SMEM)
    return fail(BQ_EUNSUPPORTED, "tile %d needs more shared memory than a CTA has", tile);
  CUDA_TRY(cudaMemcpy(s->pool + s->L.off_work, work.data(), work.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
  s->n_work = (int)work.size();
  s->smem_bytes = (int)(smem * cs);
  s->adj_smem = (int)(adj * cs);
  s->tile = tile;
  s->gread_sched = gread;
  int g = 0;
  for (const WorkItem& w : work) g = g || w.gread;
  s->has_gread = g;
  drop_graph(s);
  return BQ_OK;
}

extern "C" int bq_get_tune(const bq_state* s, bq_tune* out) {
  if (!s || !out) return fail(BQ_EINVAL, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->stage_path = s->use_pipe ? BQ_PATH_PIPE : (s->use_m1 ? BQ_PATH_SYSTEM : BQ_PATH_TILED);
  out->pipe_slots = s->pipe_nslots[0];
  out->pipe_ctas_per_sm = s->pipe_cap;
  out->solve_kernel = s->solve_ok && !s->solve_via_step ? (s->solve_mg ? BQ_SOLVE_MERGED : BQ_SOLVE_PROGRAM) : BQ_SOLVE_STEP;
  out->solve_ctas_per_sm = s->solve_cap;
  out->n_candidates = s->tune_n;
  out->step_us = s->tune_step_us;
  out->solve_us = s->tune_solve_us;
  out->tile = s->tile;
  out->lanes = s->lanes;
  out->gread = s->gread_sched;
  out->grad_coop = s->grad_coop;
  out->grad_us = s->tune_grad_us;
  out->pipe_fused = s->pipe_fused;
  return BQ_OK;
}

extern "C" int bq_set_tune(bq_state* s, const bq_tune* t) {
  if (!s || !t) return fail(BQ_EINVAL, "NULL argument");
  if (t->pipe_ctas_per_sm < 0 || t->solve_ctas_per_sm < 0) return fail(BQ_EINVAL, "negative CTA count");
  if (t->lanes != 0 && t->lanes != 1 && t->lanes != 2 && t->lanes != 4)
    return fail(BQ_EINVAL, "lanes must be 0, 1, 2 or 4");
  switch (t->stage_path) {
    case BQ_PATH_PIPE: {
      if (!s->pipe_ok) return fail(BQ_EUNSUPPORTED, "the pipelined path is not available for this state");
      const int rc = pipe_configure(s, t->pipe_slots, t->pipe_ctas_per_sm);
      if (rc != BQ_OK) return rc;
      s->use_pipe = 1;
      break;
    }
    case BQ_PATH_SYSTEM:
      if (!s->use_m1) return fail(BQ_EUNSUPPORTED, "the one-CTA-per-system path needs a single-mode state");
      s->use_pipe = 0;
      break;
    case BQ_PATH_TILED: {
      if (s->use_m1) return fail(BQ_EUNSUPPORTED, "single-mode states have no tiled work items");
      if (t->tile != s->tile || (t->gread != 0) != (s->gread_sched != 0)) {
        const int rc = apply_tile(s, t->tile, t->gread != 0);
        if (rc != BQ_OK) return rc;
      }
      break;
    }
    default:
      return fail(BQ_EINVAL, "unknown stage path %d", t->stage_path);
  }
  if (s->solve_ok) {
    if (t->solve_kernel == BQ_SOLVE_MERGED) {
      if (!s->solve_mg_ok) return fail(BQ_EUNSUPPORTED, "the merged persistent solve is not available");
      s->solve_mg = 1;
      s->solve_via_step = 0;
    } else if (t->solve_kernel == BQ_SOLVE_PROGRAM) {
      s->solve_mg = 0;
      s->solve_via_step = 0;
    } else if (t->solve_kernel == BQ_SOLVE_STEP) {
      s->solve_via_step = 1;
    } else {
      return fail(BQ_EINVAL, "unknown solve kernel %d", t->solve_kernel);
    }
    s->solve_cap = t->solve_ctas_per_sm;
  }
  s->lanes = t->lanes == 0 ? default_lanes(s->sys) : t->lanes;
  s->grad_coop = t->grad_coop != 0;
  s->pipe_fused = t->pipe_fused != 0;
  drop_graph(s);
  return BQ_OK;
}

extern "C" int bq_autotune_scratch_bytes(const bq_state* s, size_t* out) {
  if (!s || !out) return fail(BQ_EINVAL, "NULL argument");
  *out = 2 * (size_t)s->total_elems * (s->dtype == BQ_F64 ? 16 : 8);
  return BQ_OK;
}

// Tiles (with global reads) that give at most k work items per SM, k = 1, 2, 3: the smallest
// such tile for each k.  A stage then puts the same number of items on every SM instead of one
// more on some, and the SM with the most items sets the stage's time.
static std::vector<int> sm_aligned_tiles(const bq_state* s) {
  std::vector<int> out;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return out;
  const size_t cs = s->dtype == BQ_F64 ? 16 : 8;
  auto items = [&](int tl) {
    std::vector<WorkItem> w;
    int sm = 0, ad = 0;
    build_work(s->sys, cs, tl, 1, w, sm, ad);
    return (int)w.size();
  };
  int64_t max_pts = 32;
  for (const SysDesc& sd : s->sys) max_pts = std::max<int64_t>(max_pts, sd.has_r ? sd.n_r : 0);
  for (int k = 1; k <= 3; ++k) {
    int lo = 32, hi = (int)std::min<int64_t>(max_pts, 1 << 20);
    if (items(hi) > k * nsm) continue;  // even whole systems are more items than that
    while (lo < hi) {                   // smallest tile with at most k * nsm items
      const int mid = lo + (hi - lo) / 2;
      if (items(mid) <= k * nsm) hi = mid; else lo = mid + 1;
    }
    if (std::find(out.begin(), out.end(), lo) == out.end()) out.push_back(lo);
  }
  return out;
}

extern "C" int bq_autotune(bq_state* s, double dt, int trial_steps, void* scratch, size_t scratch_bytes, void* stream,
                           bq_tune* out) {
  if (!s || !scratch) return fail(BQ_EINVAL, "NULL argument");
  if (trial_steps < 1) return fail(BQ_EINVAL, "trial_steps < 1");
  if (!(dt > 0.0)) return fail(BQ_EINVAL, "dt must be > 0");
  if (dt > s->dt_max * (1.0 + 1e-12))
    return fail(BQ_EUNSTABLE_DT, "dt=%g above the RK4 stability bound %g", dt, s->dt_max);
  const size_t n = (size_t)s->total_elems * (s->dtype == BQ_F64 ? 16 : 8);
  if (scratch_bytes < 2 * n) return fail(BQ_ENOMEM, "scratch has %zu bytes, needs %zu", scratch_bytes, 2 * n);
  cudaStream_t st = (cudaStream_t)stream;
  char* b = s->pool;
  char* sc = (char*)scratch;
  const double tau0 = s->tau;
  CUDA_TRY(ensure_comp(s, st));  // the saved copy is valid for every schedule
  CUDA_TRY(cudaMemcpyAsync(sc, b + s->L.off_y, n, cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(sc + n, b + s->L.off_comp, n, cudaMemcpyDeviceToDevice, st));
  auto restore = [&]() -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(b + s->L.off_y, sc, n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + s->L.off_comp, sc + n, n, cudaMemcpyDeviceToDevice, st);
    s->obs_valid = 0;
    s->tau = tau0;
    s->tau_base_host = tau0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + s->L.off_ctrl, &s->tau_base_host, sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b + s->L.off_ctrl + 8, 0, 16, st);
    return e;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  // device time per RK4 step of `run` (after one warm-up step), with the state restored
  // before and after
  auto measure = [&](bool solve, double* us) -> int {
    for (int rep = 0; rep < 2; ++rep) {
      CUDA_TRY(restore());
      if (rep == 1) CUDA_TRY(cudaEventRecord(e0, st));
      const int64_t ns = rep == 0 ? 1 : trial_steps;
      CUDA_TRY(solve ? enqueue_solve(s, dt, ns, st) : enqueue_steps(s, dt, ns, st));
      g_launches += solve ? 1 : ns * kernels_per_step(s);
      if (rep == 1) CUDA_TRY(cudaEventRecord(e1, st));
    }
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    unsigned int err = 0;
    CUDA_TRY(cudaMemcpy(&err, b + s->L.off_ctrl + 32, sizeof(err), cudaMemcpyDeviceToHost));
    if (err) return fail(BQ_ETIMEOUT, "a bounded device wait gave up during tuning");
    *us = 1000.0 * ms / trial_steps;
    return BQ_OK;
  };
  int rc = BQ_OK;
  int ntried = 0;
  // ---- bq_step schedules --------------------------------------------------------------
  bq_tune best;
  bq_get_tune(s, &best);
  double best_step = 1e300;
  {
    struct Cand { int path, slots, cap, lanes, gread; };
    std::vector<Cand> cands;
    if (s->pipe_ok) {
      for (int slots = 2; slots <= 4; ++slots) {
        if (pipe_configure(s, slots, 0) != BQ_OK) break;
        // the occupancy limit and one CTA per SM fewer (less shared-memory and L2 pressure)
        int dev = 0, nsm = 0;
        CUDA_TRY(cudaGetDevice(&dev));
        CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const int per_sm = (s->pipe_grid[1] + nsm - 1) / nsm;
        cands.push_back({BQ_PATH_PIPE, slots, 0, 1, 0});
        if (per_sm > 2 && s->n_sys > per_sm * nsm) cands.push_back({BQ_PATH_PIPE, slots, per_sm - 1, 1, 0});
      }
    }
    if (s->use_m1) {
      cands.push_back({BQ_PATH_SYSTEM, 0, 0, 1, 0});
    } else {  // tile lengths (the cap field carries the tile; 0 = default) x lanes per point,
              // with halo windows and with global reads
      for (int tl : {0, 64, 96, 128, 192, 256, 512})
        for (int ln : {1, 2, 4}) cands.push_back({BQ_PATH_TILED, 0, tl, ln, 0});
      for (int tl : {32, 64, 128, 256, 512})
        for (int ln : {1, 2, 4}) cands.push_back({BQ_PATH_TILED, 0, tl, ln, 1});
      for (int tl : sm_aligned_tiles(s))
        for (int ln : {1, 2, 4}) cands.push_back({BQ_PATH_TILED, 0, tl, ln, 1});
    }
    const int lanes0 = s->lanes;
    for (const Cand& c : cands) {
      if (c.path == BQ_PATH_PIPE) {
        if ((rc = pipe_configure(s, c.slots, c.cap)) != BQ_OK) break;
        s->use_pipe = 1;
      } else if (c.path == BQ_PATH_TILED) {
        if ((c.cap != s->tile || c.gread != s->gread_sched) && apply_tile(s, c.cap, c.gread) != BQ_OK) {
          g_err.clear();  // a tile that does not fit
          continue;
        }
        s->lanes = c.lanes;
      } else {
        s->use_pipe = 0;
      }
      double us = 0.0;
      if ((rc = measure(false, &us)) != BQ_OK) break;
      ++ntried;
      if (us < best_step) {
        best_step = us;
        best.stage_path = c.path;
        best.pipe_slots = c.path == BQ_PATH_PIPE ? c.slots : 2;
        best.pipe_ctas_per_sm = c.path == BQ_PATH_PIPE ? c.cap : 0;
        best.tile = c.path == BQ_PATH_TILED ? c.cap : s->tile;
        best.lanes = c.path == BQ_PATH_TILED ? c.lanes : lanes0;
        best.gread = c.path == BQ_PATH_TILED ? c.gread : s->gread_sched;
      }
    }
    s->lanes = lanes0;
  }
  // ---- bq_solve schedules -------------------------------------------------------------
  double best_solve = 0.0;
  if (rc == BQ_OK && s->solve_ok) {
    best_solve = 1e300;
    const int kinds[2] = {BQ_SOLVE_MERGED, BQ_SOLVE_PROGRAM};
    for (int kind : kinds) {
      if (kind == BQ_SOLVE_MERGED && !s->solve_mg_ok) continue;
      s->solve_mg = kind == BQ_SOLVE_MERGED;
      int per_sm = 0;
      CUDA_TRY(bq::solve_blocks_per_sm(s->dtype, s->solve_mg, s->solve_mg ? s->solve_mg_smem : s->solve_smem, &per_sm));
      for (int cap : {0, per_sm - 1}) {
        if (cap < 0 || (cap == 0 && per_sm < 1) || (cap > 0 && cap >= per_sm)) continue;
        s->solve_cap = cap;
        double us = 0.0;
        if ((rc = measure(true, &us)) != BQ_OK) break;
        ++ntried;
        if (us < best_solve) {
          best_solve = us;
          best.solve_kernel = kind;
          best.solve_ctas_per_sm = cap;
        }
      }
      if (rc != BQ_OK) break;
    }
  }
  // bq_solve steps with bq_step's schedule when that was faster than every persistent kernel
  if (rc == BQ_OK && s->solve_ok && best_step < best_solve) best.solve_kernel = BQ_SOLVE_STEP;
  cudaError_t er = restore();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != BQ_OK) return rc;
  if (er != cudaSuccess) return fail(BQ_ECUDA, "restore: %s", cudaGetErrorString(er));
  CUDA_TRY(cudaStreamSynchronize(st));
  if ((rc = bq_set_tune(s, &best)) != BQ_OK) return rc;
  s->tune_n = ntried;
  s->tune_step_us = best_step;
  s->tune_solve_us = best_solve;
  if (out) bq_get_tune(s, out);
  return BQ_OK;
}


static int run_eval(bq_state* s, int g0, int n, int small, double* out_host, cudaStream_t st);

// ---------------------------------------------------------------------------------------
// Gradients (discrete adjoint with checkpointing).
// ---------------------------------------------------------------------------------------
struct GradLayout {
  size_t ckpt, rec, lam, lacc, ba, bb, srcred, grad, total;
  size_t rec_seg;  // bytes of one segment's recorded stage inputs (4 k states)
  int64_t n_ckpt;
};

static GradLayout grad_layout(const bq_state* s, int64_t n_steps, int k) {
  GradLayout g{};
  const size_t cs = s->dtype == BQ_F64 ? 16 : 8;
  const size_t arr = (size_t)s->total_elems * cs;
  size_t o = 0;
  auto seg = [&](size_t bytes) { size_t r = o; o = align_up(o + std::max<size_t>(bytes, 1)); return r; };
  g.n_ckpt = (n_steps + k - 1) / k;
  g.rec_seg = 4 * arr * (size_t)k;
  g.ckpt = seg(2 * arr * (size_t)g.n_ckpt);
  g.lam = seg(arr);
  g.lacc = seg(arr);
  g.ba = seg(arr);
  g.bb = seg(arr);
  g.srcred = seg((size_t)s->n_sys * std::max(1, s->srcred_stride) * cs);
  g.grad = seg((size_t)std::max(1, s->grad_size) * sizeof(double));
  // two segments' stage inputs (recompute overlaps the backward sweep), last: a larger
  // workspace holds further recordings (bq_grad records that many segments in its forward
  // pass and does not recompute them)
  g.rec = seg(2 * g.rec_seg);
  g.total = o;
  return g;
}

extern "C" int bq_grad_size(const bq_state* s, int* n) {
  if (!s || !n) return fail(BQ_EINVAL, "NULL argument");
  *n = s->grad_size;
  return BQ_OK;
}

extern "C" int bq_grad_required_bytes(const bq_state* s, int64_t n_steps, int checkpoint_every, size_t* out) {
  if (!s || !out || n_steps < 1 || checkpoint_every < 1) return fail(BQ_EINVAL, "bad argument");
  *out = grad_layout(s, n_steps, checkpoint_every).total;
  return BQ_OK;
}

extern "C" int bq_grad_record_bytes(const bq_state* s, int64_t n_steps, int checkpoint_every, size_t* per_segment,
                                    int64_t* n_segments) {
  if (!s || !per_segment || !n_segments || n_steps < 1 || checkpoint_every < 1) return fail(BQ_EINVAL, "bad argument");
  const GradLayout G = grad_layout(s, n_steps, checkpoint_every);
  *per_segment = G.rec_seg;
  *n_segments = G.n_ckpt;
  return BQ_OK;
}

static cudaError_t enqueue_steps_rec(bq_state* s, double dt, int64_t n, cudaStream_t st, char* rec, size_t arr) {
  for (int64_t i = 0; i < n; ++i)
    for (int stage = 1; stage <= 4; ++stage) {
      bq::StageArgs a = stage_args(s, stage, dt);
      a.rec = rec ? rec + ((size_t)i * 4 + stage - 1) * arr : nullptr;
      cudaError_t e = launch_any_stage(s, a, st);
      if (e != cudaSuccess) return e;
      g_launches += kernels_per_stage(s, a.rec != nullptr);
    }
  return cudaSuccess;
}

static int set_tau(bq_state* s, double tau, cudaStream_t st) {
  s->tau = tau;
  s->tau_base_host = tau;
  CUDA_TRY(cudaMemcpyAsync(s->pool + s->L.off_ctrl, &s->tau_base_host, sizeof(double), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemsetAsync(s->pool + s->L.off_ctrl + 8, 0, 16, st));
  CUDA_TRY(cudaStreamSynchronize(st));  // the host value above is reused immediately
  return BQ_OK;
}

extern "C" int bq_grad(bq_state* s, double dt, int64_t n_steps, int checkpoint_every, void* work, size_t work_bytes,
                       double* loss_out, double* grad_out, void* stream) {
  if (!s || !work || !loss_out || !grad_out) return fail(BQ_EINVAL, "NULL argument");
  if (n_steps < 1 || checkpoint_every < 1 || !(dt > 0.0)) return fail(BQ_EINVAL, "bad step arguments");
  if (dt > s->dt_max * (1.0 + 1e-12)) return fail(BQ_EUNSTABLE_DT, "dt=%g above the RK4 bound %g", dt, s->dt_max);
  const GradLayout G = grad_layout(s, n_steps, checkpoint_every);
  if (work_bytes < G.total) return fail(BQ_ENOMEM, "gradient workspace has %zu bytes, needs %zu", work_bytes, G.total);
  if (((uintptr_t)work & 255) != 0) return fail(BQ_EINVAL, "gradient workspace must be 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)work;
  char* b = s->pool;
  const Layout& L = s->L;
  const size_t cs = s->dtype == BQ_F64 ? 16 : 8;
  const size_t arr = (size_t)s->total_elems * cs;
  const double tau0 = s->tau;
  const int k = checkpoint_every;
  CUDA_TRY(cudaMemsetAsync(w + G.grad, 0, (size_t)std::max(1, s->grad_size) * sizeof(double), st));
  // Cooperative segment kernels (tiled path): one launch per segment and direction, grids of
  // at most the resident CTAs and no more than the largest phase's items.
  int grid_f = 0, grid_b = 0;
  if (s->grad_coop && !s->use_m1) {
    CUDA_TRY(bq::coop_max_grid(s->dtype, s->nm, false, s->smem_bytes, &grid_f));
    CUDA_TRY(bq::coop_max_grid(s->dtype, s->nm, true, s->adj_smem, &grid_b));
    const int src_items = s->max_s > 0 ? s->n_sys * s->max_s * 2 * ((s->ng_max + 3) / 4) : 0;  // BQ_SRC_TILE_COOP
    grid_f = std::min(grid_f, s->n_work);
    grid_b = std::min(grid_b, std::max(s->n_work, src_items));
  }
  const bool coop = grid_f > 0 && grid_b > 0;
  // Recording buffers: the two of the layout plus as many more as the workspace holds.  On
  // the cooperative path the forward pass records the last n_rec segments, which the
  // backward sweep then does not recompute; segment c uses buffer c % n_rec.
  int64_t n_rec = 2 + (int64_t)((work_bytes - G.total) / G.rec_seg);
  n_rec = std::max<int64_t>(1, std::min<int64_t>(n_rec, G.n_ckpt));
  auto rec_buf = [&](int64_t c) { return w + G.rec + (size_t)(c % n_rec) * G.rec_seg; };
  auto recorded = [&](int64_t c) { return coop && c >= G.n_ckpt - n_rec; };
  bq::CoopArgs P;
  std::memset(&P, 0, sizeof(P));
  if (coop) {
    P.st = stage_args(s, 1, dt);
    P.ua = b + L.off_ua;
    P.ub = b + L.off_ub;
    P.arr = arr;
    P.n_work = s->n_work;
    P.n_sys = s->n_sys;
    P.max_s = s->max_s;
    P.bar = (unsigned int*)(b + L.off_ctrl + 48);
    P.error = (unsigned int*)(b + L.off_ctrl + 32);
  }
  auto coop_fwd = [&](double tau_seg, int64_t n, char* rec, cudaStream_t cs) -> cudaError_t {
    P.tau0 = tau_seg;
    P.n_steps = (int)n;
    P.rec = rec;
    cudaError_t e = cudaMemsetAsync(P.bar, 0, 8, cs);
    if (e == cudaSuccess) e = bq::launch_coop(s->dtype, s->nm, false, P, s->smem_bytes, grid_f, cs);
    g_launches++;
    return e;
  };
  // ---- forward with checkpoints ----------------------------------------------------------
  // (checkpoints hold the folded form: the recording stage kernels start from them)
  for (int64_t c = 0; c < G.n_ckpt; ++c) {
    const int64_t n0 = c * k, n1 = std::min<int64_t>(n_steps, n0 + k);
    CUDA_TRY(ensure_comp(s, st));
    CUDA_TRY(cudaMemcpyAsync(w + G.ckpt + (2 * c) * arr, b + L.off_y, arr, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(w + G.ckpt + (2 * c + 1) * arr, b + L.off_comp, arr, cudaMemcpyDeviceToDevice, st));
    if (coop) {
      CUDA_TRY(coop_fwd(tau0 + (double)n0 * dt, n1 - n0, recorded(c) ? rec_buf(c) : nullptr, st));
      continue;
    }
    int r = set_tau(s, tau0 + (double)n0 * dt, st);
    if (r != BQ_OK) return r;
    CUDA_TRY(enqueue_steps_rec(s, dt, n1 - n0, st, nullptr, arr));
  }
  s->tau = tau0 + (double)n_steps * dt;
  CUDA_TRY(ensure_comp(s, st));
  // ---- loss and the cotangent of the final state -----------------------------------------
  std::vector<double> tr(2 * (size_t)s->B);
  int r = run_eval(s, 0, s->n_trace_groups, s->trace_small, tr.data(), st);
  if (r != BQ_OK) return r;
  for (int i = 0; i < s->B; ++i) loss_out[i] = tr[2 * i];
  CUDA_TRY(cudaMemsetAsync(w + G.lam, 0, arr, st));
  CUDA_TRY(bq::launch_adj_seed((const SysDesc*)(b + L.off_sys), (const EvalGroup*)(b + L.off_groups),
                               (const EvalEntry*)(b + L.off_entries), b + L.off_y, w + G.lam, s->n_trace_groups,
                               s->dtype, st));
  g_launches++;
  // ---- backward sweep ----------------------------------------------------------------------
  if (coop) {
    // per segment, last first: restore its checkpoint, one cooperative launch recomputes it
    // recording every stage input, one runs its adjoint (all on the caller's stream)
    P.adj.sys = (const SysDesc*)(b + L.off_sys);
    P.adj.terms = (const TermDesc*)(b + L.off_terms);
    P.adj.chans = (const ChanDesc*)(b + L.off_chans);
    P.adj.chpar = (const double*)(b + L.off_chpar);
    P.adj.wtab = b + L.off_wtab;
    P.adj.diag = b + L.off_diag;
    P.adj.work = (const WorkItem*)(b + L.off_work);
    P.adj.dc = (const double2*)(b + L.off_dc);
    P.adj.srcred = w + G.srcred;
    P.adj.grad = (double*)(w + G.grad);
    P.adj.dt = dt;
    P.adj.horizon = s->horizon;
    P.adj.reverse = s->reverse;
    P.adj.srcred_stride = s->srcred_stride;
    P.adj.ng_max = s->ng_max;
    P.adj.lanes = s->lanes;
    P.ba = w + G.ba;
    P.bb = w + G.bb;
    char* lam = w + G.lam;
    char* lacc = w + G.lacc;
    for (int64_t c = G.n_ckpt - 1; c >= 0; --c) {
      const int64_t n0 = c * k, n1 = std::min<int64_t>(n_steps, n0 + k);
      char* rec = rec_buf(c);
      if (!recorded(c)) {
        CUDA_TRY(cudaMemcpyAsync(b + L.off_y, w + G.ckpt + (2 * c) * arr, arr, cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(b + L.off_comp, w + G.ckpt + (2 * c + 1) * arr, arr, cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(coop_fwd(tau0 + (double)n0 * dt, n1 - n0, rec, st));
      }
      P.tau0 = tau0 + (double)n0 * dt;  // (the recomputation, when it runs, sets the same)
      P.n_steps = (int)(n1 - n0);
      P.rec = rec;
      P.lam = lam;
      P.lacc = lacc;
      CUDA_TRY(cudaMemsetAsync(P.bar, 0, 8, st));
      CUDA_TRY(bq::launch_coop(s->dtype, s->nm, true, P, s->adj_smem, grid_b, st));
      g_launches++;
      if ((n1 - n0) & 1) std::swap(lam, lacc);
    }
  } else {
  // Segment c is recomputed from its checkpoint (recording every stage input into buffer
  // c % 2) on one stream while the adjoint of segment c + 1 runs on another: the two chains
  // are independent until the adjoint of c needs the recording of c, and the recomputation of
  // c - 1 reuses the buffer of c + 1 only after that segment's adjoint has finished.
  for (cudaStream_t& gs : s->grad_stream)
    if (!gs) CUDA_TRY(cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
  cudaStream_t sF = s->grad_stream[0], sB = s->grad_stream[1];
  cudaEvent_t ev[6] = {};  // start, recorded[2], adjoint done[2], end
  for (cudaEvent_t& e : ev) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() { for (int i = 0; i < 6; ++i) if (e[i]) cudaEventDestroy(e[i]); }
  } ev_guard{ev};
  CUDA_TRY(cudaEventRecord(ev[0], st));
  CUDA_TRY(cudaStreamWaitEvent(sF, ev[0], 0));
  CUDA_TRY(cudaStreamWaitEvent(sB, ev[0], 0));
  const size_t rec_bytes = 4 * arr * (size_t)k;
  char* lam = w + G.lam;
  char* lacc = w + G.lacc;
  bq::AdjArgs a;
  std::memset(&a, 0, sizeof(a));
  a.sys = (const SysDesc*)(b + L.off_sys);
  a.terms = (const TermDesc*)(b + L.off_terms);
  a.chans = (const ChanDesc*)(b + L.off_chans);
  a.chpar = (const double*)(b + L.off_chpar);
  a.wtab = b + L.off_wtab;
  a.diag = b + L.off_diag;
  a.work = (const WorkItem*)(b + L.off_work);
  a.dc = (const double2*)(b + L.off_dc);
  a.srcred = w + G.srcred;
  a.grad = (double*)(w + G.grad);
  a.dt = dt;
  a.horizon = s->horizon;
  a.reverse = s->reverse;
  a.srcred_stride = s->srcred_stride;
  a.ng_max = s->ng_max;
  a.lanes = s->lanes;
  for (int64_t c = G.n_ckpt - 1; c >= 0; --c) {
    const int64_t n0 = c * k, n1 = std::min<int64_t>(n_steps, n0 + k);
    const int buf = (int)(c & 1);
    char* rec = w + G.rec + (size_t)buf * rec_bytes;
    // recompute the segment from its checkpoint, recording every stage input
    if (c + 2 < G.n_ckpt) CUDA_TRY(cudaStreamWaitEvent(sF, ev[3 + buf], 0));  // adjoint of c + 2 is done with the buffer
    CUDA_TRY(cudaMemcpyAsync(b + L.off_y, w + G.ckpt + (2 * c) * arr, arr, cudaMemcpyDeviceToDevice, sF));
    CUDA_TRY(cudaMemcpyAsync(b + L.off_comp, w + G.ckpt + (2 * c + 1) * arr, arr, cudaMemcpyDeviceToDevice, sF));
    r = set_tau(s, tau0 + (double)n0 * dt, sF);
    if (r != BQ_OK) return r;
    CUDA_TRY(enqueue_steps_rec(s, dt, n1 - n0, sF, rec, arr));
    CUDA_TRY(cudaEventRecord(ev[1 + buf], sF));
    CUDA_TRY(cudaStreamWaitEvent(sB, ev[1 + buf], 0));
    for (int64_t n = n1 - 1; n >= n0; --n) {
      a.tau_step = tau0 + (double)n * dt;
      a.lam = lam;
      a.lacc = lacc;
      for (int stage = 4; stage >= 1; --stage) {
        a.stage = stage;
        a.u = rec + ((size_t)(n - n0) * 4 + stage - 1) * arr;
        a.b_in = stage == 4 ? nullptr : (stage == 3 ? (void*)(w + G.ba) : (stage == 2 ? (void*)(w + G.bb) : (void*)(w + G.ba)));
        a.b_out = stage == 4 ? (void*)(w + G.ba) : (stage == 3 ? (void*)(w + G.bb) : (stage == 2 ? (void*)(w + G.ba) : nullptr));
        CUDA_TRY(bq::launch_adjoint(a, s->dtype, s->nm, s->n_work, s->adj_smem, s->n_sys, s->max_s, sB));
        g_launches += s->max_s > 0 ? 2 : 1;
      }
      std::swap(lam, lacc);
    }
    CUDA_TRY(cudaEventRecord(ev[3 + buf], sB));
  }
  // join both streams into the caller's
  CUDA_TRY(cudaEventRecord(ev[5], sB));
  CUDA_TRY(cudaStreamWaitEvent(st, ev[5], 0));
  CUDA_TRY(cudaEventRecord(ev[1], sF));
  CUDA_TRY(cudaStreamWaitEvent(st, ev[1], 0));
  }
  // leave the state as it was before the call (initial content, tau0)
  s->obs_valid = 0;
  CUDA_TRY(cudaMemcpyAsync(b + L.off_y, w + G.ckpt, arr, cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(b + L.off_comp, w + G.ckpt + arr, arr, cudaMemcpyDeviceToDevice, st));
  r = set_tau(s, tau0, st);
  if (r != BQ_OK) return r;
  CUDA_TRY(cudaMemcpyAsync(grad_out, w + G.grad, (size_t)s->grad_size * sizeof(double), cudaMemcpyDeviceToHost, st));
  unsigned int err_word = 0;
  CUDA_TRY(cudaMemcpyAsync(&err_word, b + L.off_ctrl + 32, sizeof(err_word), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (err_word) return fail(BQ_ETIMEOUT, "a bounded device wait gave up during the gradient (error word %u)", err_word);
  for (int i = 0; i < s->grad_size; ++i)
    if (!std::isfinite(grad_out[i])) return fail(BQ_ENONFINITE, "non-finite gradient");
  return BQ_OK;
}

extern "C" int bq_autotune_grad(bq_state* s, double dt, int trial_steps, int checkpoint_every, void* work,
                                size_t work_bytes, void* stream, bq_tune* out) {
  if (!s || !work) return fail(BQ_EINVAL, "NULL argument");
  if (trial_steps < 1 || checkpoint_every < 1) return fail(BQ_EINVAL, "bad trial arguments");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<double> loss(s->B), g(std::max(1, s->grad_size));
  struct Cand { int tile, lanes, gread; };
  std::vector<Cand> cands;
  if (s->use_m1) {
    for (int ln : {1, 2, 4}) cands.push_back({s->tile, ln, s->gread_sched});
  } else {
    for (int gr : {0, 1})
      for (int tl : {0, 32, 64, 96, 128, 192, 256, 512})
        for (int ln : {1, 2, 4}) cands.push_back({tl, ln, gr});
    // tiles that give at most k work items per SM (the FP64 stages are bound by each SM's
    // FP64 pipe, so the SM with the most items sets the stage's time)
    for (int tl : sm_aligned_tiles(s)) {
      bool have = false;
      for (const Cand& c : cands) have = have || (c.tile == tl && c.gread == 1);
      if (!have)
        for (int ln : {1, 2, 4}) cands.push_back({tl, ln, 1});
    }
  }
  const int tile0 = s->tile, lanes0 = s->lanes, gread0 = s->gread_sched;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } guard{e0, e1};
  double best_us = 1e300;
  Cand best{tile0, lanes0, gread0};
  int ntried = 0;
  for (const Cand& c : cands) {
    if (!s->use_m1 && (c.tile != s->tile || c.gread != s->gread_sched) && apply_tile(s, c.tile, c.gread) != BQ_OK) {
      g_err.clear();  // a tile that does not fit
      continue;
    }
    s->lanes = c.lanes;
    int rc = bq_grad(s, dt, std::min(trial_steps, checkpoint_every), checkpoint_every, work, work_bytes, loss.data(),
                     g.data(), stream);  // warm-up
    if (rc == BQ_OK) {
      CUDA_TRY(cudaEventRecord(e0, st));
      rc = bq_grad(s, dt, trial_steps, checkpoint_every, work, work_bytes, loss.data(), g.data(), stream);
      CUDA_TRY(cudaEventRecord(e1, st));
    }
    if (rc != BQ_OK) {
      // restore the schedule the state had, then report
      if (!s->use_m1) apply_tile(s, tile0, gread0);
      s->lanes = lanes0;
      return rc;
    }
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    const double us = 1000.0 * ms / trial_steps;
    ++ntried;
    if (us < best_us) { best_us = us; best = c; }
  }
  if (!s->use_m1 && (best.tile != s->tile || best.gread != s->gread_sched)) {
    const int rc = apply_tile(s, best.tile, best.gread);
    if (rc != BQ_OK) return rc;
  }
  s->lanes = best.lanes;
  s->tune_grad_us = best_us;
  drop_graph(s);
  if (out) {
    bq_get_tune(s, out);
    out->n_candidates = ntried;
  }
  return BQ_OK;
}

extern "C" int bq_time(const bq_state* s, double* tau) {
  if (!s || !tau) return fail(BQ_EINVAL, "NULL argument");
  *tau = s->tau;
  return BQ_OK;
}

// ---------------------------------------------------------------------------------------
// Evaluation.
// ---------------------------------------------------------------------------------------
static int run_eval(bq_state* s, int g0, int n, int small, double* out_host, cudaStream_t st) {
  char* b = s->pool;
  const Layout& L = s->L;
  CUDA_TRY(ensure_comp(s, st));
  CUDA_TRY(bq::launch_eval((const SysDesc*)(b + L.off_sys), (const EvalGroup*)(b + L.off_groups) + g0,
                           (const EvalEntry*)(b + L.off_entries), b + L.off_y, b + L.off_comp,
                           (double2*)(b + L.off_out) + g0, n,
                           s->dtype, small, st));
  g_launches++;
  CUDA_TRY(cudaMemcpyAsync(out_host, b + L.off_out + (size_t)g0 * 16, (size_t)n * 16, cudaMemcpyDeviceToHost, st));
  unsigned int err_word = 0;
  CUDA_TRY(cudaMemcpyAsync(&err_word, b + L.off_ctrl + 32, sizeof(err_word), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (err_word) return fail(BQ_ETIMEOUT, "a bounded device wait gave up during stepping (error word %u)", err_word);
  for (int i = 0; i < 2 * n; ++i)
    if (!std::isfinite(out_host[i])) return fail(BQ_ENONFINITE, "non-finite observable");
  return BQ_OK;
}

// Enqueues Tr(rho0_b A_b) of every problem into the pool's output slots: from the per-system
// contributions of the last pipelined stage 4 when they describe the current state, else
// with the evaluation kernel.
static int enqueue_trace(bq_state* s, cudaStream_t st) {
  char* b = s->pool;
  const Layout& L = s->L;
  if (s->obs_valid) {
    CUDA_TRY(bq::launch_obs_sum((const double2*)(b + L.off_obs), (const EvalGroup*)(b + L.off_groups),
                                s->n_trace_groups, (double2*)(b + L.off_out), st));
    g_launches++;
    return BQ_OK;
  }
  CUDA_TRY(ensure_comp(s, st));
  CUDA_TRY(bq::launch_eval((const SysDesc*)(b + L.off_sys), (const EvalGroup*)(b + L.off_groups),
                           (const EvalEntry*)(b + L.off_entries), b + L.off_y, b + L.off_comp,
                           (double2*)(b + L.off_out), s->n_trace_groups, s->dtype, s->trace_small, st));
  g_launches++;
  return BQ_OK;
}

extern "C" int bq_evaluate(bq_state* s, double* out_host, void* stream) {
  if (!s || !out_host) return fail(BQ_EINVAL, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int n = s->n_trace_groups;
  int r = enqueue_trace(s, st);
  if (r != BQ_OK) return r;
  CUDA_TRY(cudaMemcpyAsync(out_host, s->pool + s->L.off_out, (size_t)n * 16, cudaMemcpyDeviceToHost, st));
  unsigned int err_word = 0;
  CUDA_TRY(cudaMemcpyAsync(&err_word, s->pool + s->L.off_ctrl + 32, sizeof(err_word), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (err_word) return fail(BQ_ETIMEOUT, "a bounded device wait gave up during stepping (error word %u)", err_word);
  for (int i = 0; i < 2 * n; ++i)
    if (!std::isfinite(out_host[i])) return fail(BQ_ENONFINITE, "non-finite observable of problem %d", i / 2);
  return BQ_OK;
}

extern "C" int bq_evaluate_async(bq_state* s, double* out, void* stream) {
  if (!s || !out) return fail(BQ_EINVAL, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  int r = enqueue_trace(s, st);
  if (r != BQ_OK) return r;
  CUDA_TRY(cudaMemcpyAsync(out, s->pool + s->L.off_out, (size_t)s->n_trace_groups * 16, cudaMemcpyDefault, st));
  return BQ_OK;
}

extern "C" int bq_fock_block(bq_state* s, int lo, double* out_host, void* stream) {
  if (!s || !out_host) return fail(BQ_EINVAL, "NULL argument");
  if (s->block_dim <= 0) return fail(BQ_EUNSUPPORTED, "problems of the batch have different block shapes");
  if (lo != 3) return fail(BQ_EUNSUPPORTED, "only lo = 3 (the paper's three lowest levels) is precompiled");
  return run_eval(s, s->n_trace_groups, s->n_block_groups, s->block_small, out_host, (cudaStream_t)stream);
}

extern "C" int bq_state_info(const bq_state* s, int* n_systems, int64_t* total_elems) {
  if (!s) return fail(BQ_EINVAL, "state is NULL");
  if (n_systems) *n_systems = s->n_sys;
  if (total_elems) *total_elems = s->total_elems;
  return BQ_OK;
}

extern "C" int bq_system_info(const bq_state* s, int sys, int* problem, int* p_idx, int* q_idx, int64_t* n_gx,
                              int64_t* n_gy, int64_t* n_r, double* w, double* c) {
  if (!s || sys < 0 || sys >= s->n_sys) return fail(BQ_EINVAL, "bad system index");
  const SysDesc& sd = s->sys[sys];
  if (problem) *problem = sd.prob;
  if (p_idx) *p_idx = sd.p_flat;
  if (q_idx) *q_idx = sd.q_flat;
  if (n_gx) *n_gx = sd.has_sep ? sd.n_g : 0;
  if (n_gy) *n_gy = sd.has_sep ? sd.n_g : 0;
  if (n_r) *n_r = sd.has_r ? (sd.r_diag ? (int64_t)sd.n_g * sd.n_g : sd.n_r) : 0;  // expanded view
  if (w) { w[0] = sd.w_re; w[1] = sd.w_im; }
  if (c) { c[0] = sd.c_re; c[1] = sd.c_im; }
  return BQ_OK;
}

extern "C" int bq_read_system(bq_state* s, int sys, double* gx, double* gy, double* r, void* stream) {
  if (!s || sys < 0 || sys >= s->n_sys) return fail(BQ_EINVAL, "bad system index");
  const SysDesc& sd = s->sys[sys];
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(ensure_comp(s, st));  // y alone is then the state to rounding
  const size_t cs = s->dtype == BQ_F64 ? 16 : 8;
  const char* y = s->pool + s->L.off_y;
  const int nm = s->nm;
  auto sflat = [&](int f) {  // s(k) of the storage basis for a flat per-mode index
    double v = 1.0;
    for (int j = nm - 1; j >= 0; --j) { const int k = f % sd.M[j]; f /= sd.M[j]; v *= s_of(s->basis, k); }
    return v;
  };
  auto fetch = [&](int64_t off, int64_t n, double* dst, bool is_r) -> int {
    std::vector<char> h((size_t)n * cs);
    CUDA_TRY(cudaMemcpyAsync(h.data(), y + off * cs, (size_t)n * cs, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < n; ++i) {
      double re, im;
      if (cs == 16) { re = ((double*)h.data())[2 * i]; im = ((double*)h.data())[2 * i + 1]; }
      else { re = ((float*)h.data())[2 * i]; im = ((float*)h.data())[2 * i + 1]; }
      double sc = 1.0;
      if (s->method == BQ_METHOD_MAPPED) {
        if (is_r) sc = sflat((int)(i / sd.n_g)) * sflat((int)(i % sd.n_g));
        else sc = sflat((int)i);
      }
      dst[2 * i] = re / sc;
      dst[2 * i + 1] = im / sc;
    }
    return BQ_OK;
  };
  int rc;
  if (gx && sd.has_sep && (rc = fetch(sd.off_gx, sd.n_g, gx, false)) != BQ_OK) return rc;
  if (gy && sd.has_sep && (rc = fetch(sd.off_gy, sd.n_g, gy, false)) != BQ_OK) return rc;
  if (r && sd.has_r && sd.r_diag) {  // expand the k = l entries to the n_g x n_g matrix
    std::vector<double> d(2 * (size_t)sd.n_g);
    if ((rc = fetch(sd.off_r, sd.n_g, d.data(), false)) != BQ_OK) return rc;
    std::fill(r, r + 2 * (size_t)sd.n_g * sd.n_g, 0.0);
    for (int i = 0; i < sd.n_g; ++i) {
      const double sc = s->method == BQ_METHOD_MAPPED ? sflat(i) : 1.0;  // second factor of s(k) s(l)
      r[2 * ((size_t)i * sd.n_g + i)] = d[2 * i] / sc;
      r[2 * ((size_t)i * sd.n_g + i) + 1] = d[2 * i + 1] / sc;
    }
  } else if (r && sd.has_r && (rc = fetch(sd.off_r, sd.n_r, r, true)) != BQ_OK) {
    return rc;
  }
  return BQ_OK;
}

extern "C" int bq_state_bytes(const bq_state* s, size_t* nbytes) {
  if (!s || !nbytes) return fail(BQ_EINVAL, "NULL argument");
  *nbytes = (size_t)s->total_elems * (s->dtype == BQ_F64 ? 16 : 8);
  return BQ_OK;
}

extern "C" int bq_store_state(bq_state* s, void* host, void* stream) {
  if (!s || !host) return fail(BQ_EINVAL, "NULL argument");
  const size_t n = (size_t)s->total_elems * (s->dtype == BQ_F64 ? 16 : 8);
  CUDA_TRY(ensure_comp(s, (cudaStream_t)stream));  // y alone is then the state to rounding
  CUDA_TRY(cudaMemcpyAsync(host, s->pool + s->L.off_y, n, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  return BQ_OK;
}

extern "C" int bq_load_state(bq_state* s, const void* host, void* stream) {
  if (!s || !host) return fail(BQ_EINVAL, "NULL argument");
  const size_t n = (size_t)s->total_elems * (s->dtype == BQ_F64 ? 16 : 8);
  CUDA_TRY(cudaMemcpyAsync(s->pool + s->L.off_y, host, n, cudaMemcpyHostToDevice, (cudaStream_t)stream));
  // comp is cleared lazily: the next pipelined stage 1 treats it as zero, any other consumer
  // clears it first
  s->comp_zero = 1;
  s->obs_valid = 0;
  return BQ_OK;
}

extern "C" int bq_set_time(bq_state* s, double tau) {
  if (!s || !std::isfinite(tau)) return fail(BQ_EINVAL, "bad argument");
  s->tau = tau;
  return BQ_OK;
}

// ---------------------------------------------------------------------------------------
// Diagnostics.
// ---------------------------------------------------------------------------------------
extern "C" const char* bq_status_string(int status) {
  switch (status) {
    case BQ_OK: return "ok";
    case BQ_EINVAL: return "invalid argument";
    case BQ_EUNSTABLE_DT: return "time step above the RK4 stability bound";
    case BQ_ENOMEM: return "device buffer too small";
    case BQ_ECUDA: return "CUDA error";
    case BQ_ENONFINITE: return "non-finite value";
    case BQ_ETIMEOUT: return "device wait timed out";
    case BQ_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

extern "C" const char* bq_last_error(void) { return g_err.c_str(); }

extern "C" int64_t bq_launch_count(void) { return g_launches.load(); }
