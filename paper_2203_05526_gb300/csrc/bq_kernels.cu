// CUDA kernels of the mapped adjoint-Lindblad solver (sm_103a).
//
//  * k_stage     one fused classical-RK4 stage of the coupled system of Eqs. 9a-c / 303a-c
//                (or of Eq. 3 itself for the direct number-basis method): stencil terms of
//                H and of the dissipators, the separable source S(G_x G_y), and the RK4
//                combine, for every point of a tile staged in shared memory.
//  * k_eval      observables of Eqs. 7 / 11: warp reductions over initial conditions.
//  * k_scatter   initial state (Eqs. 10, 13).
//
// Memory-bound by design: the stencil has reach one per variable and ~8-12 complex terms
// per point, so it never touches the tensor cores.  Loads of the stage input are staged
// once per CTA in shared memory (halo re-reads come from there), the state, stage output
// and accumulator are streamed with coalesced accesses.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "bq_internal.h"
#include "bq_launch.h"

namespace bq {

template <typename T> struct C2T;
template <> struct C2T<double> { using type = double2; };
template <> struct C2T<float> { using type = float2; };

template <typename C> __device__ __forceinline__ C cmk(double re, double im);
template <> __device__ __forceinline__ double2 cmk<double2>(double re, double im) { return make_double2(re, im); }
template <> __device__ __forceinline__ float2 cmk<float2>(double re, double im) {
  return make_float2((float)re, (float)im);
}

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a + s * b (complex s)
template <typename C> __device__ __forceinline__ C cfma(C s, C b, C a) {
  a.x = fma(s.x, b.x, fma(-s.y, b.y, a.x));
  a.y = fma(s.x, b.y, fma(s.y, b.x, a.y));
  return a;
}
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { a.x *= s; a.y *= s; return a; }
// a + s * b (real s)
template <typename C, typename T> __device__ __forceinline__ C caxpy(T s, C b, C a) {
  a.x = fma(s, b.x, a.x); a.y = fma(s, b.y, a.y); return a;
}

// ---------------------------------------------------------------------------------------
// Drive envelopes (channel kinds of bq.h).
// ---------------------------------------------------------------------------------------
__device__ double2 chan_value(const ChanDesc& c, const double* par, double t) {
  const double* p = par + c.par_off;
  switch (c.kind) {
    case 0:  // CONST
      return make_double2(p[0], p[1]);
    case 1: {  // GAUSS
      const double d = t - p[2];
      const double e = exp(-(d * d) / (2.0 * p[3] * p[3]));
      return make_double2(p[0] * e, p[1] * e);
    }
    case 2: {  // PWC
      const int n_seg = (c.n_par - 2) / 2;
      const double x = floor((t - p[0]) / p[1]);
      if (!(x >= 0.0) || x >= (double)n_seg) return make_double2(0.0, 0.0);
      const int s = (int)x;
      return make_double2(p[2 + 2 * s], p[3 + 2 * s]);
    }
    case 3: {  // CEXP
      double sn, cs;
      sincos(p[2] * t, &sn, &cs);
      return make_double2(p[0] * cs - p[1] * sn, p[0] * sn + p[1] * cs);
    }
    default:
      return make_double2(0.0, 0.0);
  }
}

__device__ __forceinline__ double stage_c(int stage) {
  return stage == 1 ? 0.0 : (stage == 4 ? 1.0 : 0.5);
}

// Coefficient of term t at the current stage: c * [channel or its conjugate].
__device__ __forceinline__ double2 term_coef(const TermDesc& td, const ChanDesc* chans, const double* chpar,
                                             double tau_step, double dt, int stage, double horizon, int reverse) {
  double2 c = make_double2(td.c_re, td.c_im);
  if (td.ch >= 0) {
    const ChanDesc cd = chans[td.ch];
    const double tau = (cd.kind == 2) ? tau_step + 0.5 * dt : tau_step + stage_c(stage) * dt;
    const double t = reverse ? horizon - tau : tau;
    double2 e = chan_value(cd, chpar, t);
    if (td.conj) e.y = -e.y;
    c = make_double2(c.x * e.x - c.y * e.y, c.x * e.y + c.y * e.x);
  }
  return c;
}

// ---------------------------------------------------------------------------------------
// Fused RK4 stage.
// ---------------------------------------------------------------------------------------
template <typename T, int NM>
__global__ void __launch_bounds__(BQ_BLOCK) k_stage(const StageArgs A) {
  using C = typename C2T<T>::type;
  constexpr int ND = 2 * NM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* win = reinterpret_cast<C*>(smem_raw);

  __shared__ SysDesc sd;
  __shared__ WorkItem wi;
  __shared__ TermDesc st[BQ_MAX_TERMS];
  __shared__ C sc[BQ_MAX_TERMS];
  __shared__ double s_tau;

  const int tid = threadIdx.x;
  if (tid == 0) {
    wi = A.work[blockIdx.x];
    sd = A.sys[wi.sys];
    s_tau = A.tau_base[0] + (double)(*(volatile long long*)A.counter) * A.dt;
  }
  __syncthreads();
  const int nt = sd.n_terms;
  for (int t = tid; t < nt; t += blockDim.x) {
    st[t] = A.terms[sd.term_off + t];
    const double2 c = term_coef(st[t], A.chans, A.chpar, s_tau, A.dt, A.stage, A.horizon, A.reverse);
    sc[t] = cmk<C>(c.x, c.y);
  }
  // Stage the R window and (for the separable part) G_x, G_y of the stage input.
  const C* uin = reinterpret_cast<const C*>(A.u_in);
  const int wn = wi.win_hi - wi.win_lo;
  if (sd.has_r) {
    const C* src = uin + sd.off_r + wi.win_lo;
    for (int i = tid; i < wn; i += blockDim.x) win[i] = src[i];
  }
  C* gxs = win + wn;
  C* gys = gxs + sd.n_g;
  if (sd.has_sep && (wi.do_sep || sd.has_r)) {
    const C* sx = uin + sd.off_gx;
    const C* sy = uin + sd.off_gy;
    for (int i = tid; i < sd.n_g; i += blockDim.x) {
      gxs[i] = sx[i];
      gys[i] = sy[i];
    }
  }
  __syncthreads();

  const T* W = reinterpret_cast<const T*>(A.wtab);
  const C* D = reinterpret_cast<const C*>(A.diag) + sd.diag_off;
  C* uout = reinterpret_cast<C*>(A.u_out);
  C* y = reinterpret_cast<C*>(A.y);
  C* acc = reinterpret_cast<C*>(A.acc);
  const T dt = (T)A.dt;
  const int stage = A.stage;
  int Md[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d) Md[d] = sd.M[d % NM];
  // diag table offsets: dim d's table starts at sum_{d' < d} M_d'
  int doff[ND];
  {
    int o = 0;
#pragma unroll
    for (int d = 0; d < ND; ++d) { doff[d] = o; o += Md[d]; }
  }

  // Classical RK4 with the stage sum kept as an increment (inc = k1 + 2 k2 + 2 k3) and a
  // compensated (Kahan) update of the state at stage 4, y += dt/6 (inc + k4): in FP32 the
  // per-step increment is a few ulps of y, and adding partial increments to y four times
  // per step (or even once without compensation) biases the rounding in one direction.
  C* comp = reinterpret_cast<C*>(A.comp);
  auto combine = [&](int64_t gi, C uc, C k) {
    if (stage == 1) {
      uout[gi] = caxpy(dt * (T)0.5, k, uc);
      acc[gi] = k;
    } else if (stage == 4) {
      const C yv = y[gi];
      const C s = cadd(acc[gi], k);
      const C cv = comp[gi];
      C d, t, c2;
      d.x = dt * (T)(1.0 / 6.0) * s.x - cv.x;
      d.y = dt * (T)(1.0 / 6.0) * s.y - cv.y;
      t.x = yv.x + d.x;
      t.y = yv.y + d.y;
      c2.x = (t.x - yv.x) - d.x;
      c2.y = (t.y - yv.y) - d.y;
      y[gi] = t;
      comp[gi] = c2;
    } else {
      const C yv = y[gi];
      uout[gi] = caxpy(stage == 2 ? dt * (T)0.5 : dt, k, yv);
      acc[gi] = caxpy((T)2, k, acc[gi]);
    }
  };

  // ---- R points of the tile -------------------------------------------------------
  if (sd.has_r) {
    const int ng = sd.n_g;
    for (int p = wi.start + tid; p < wi.start + wi.len; p += blockDim.x) {
      int idx[ND];
      const int kx = p / ng;
      const int ly = p - kx * ng;
      {
        int r = kx;
#pragma unroll
        for (int d = NM - 1; d >= 0; --d) { idx[d] = r % Md[d]; r /= Md[d]; }
        r = ly;
#pragma unroll
        for (int d = ND - 1; d >= NM; --d) { idx[d] = r % Md[d]; r /= Md[d]; }
      }
      const C uc = win[p - wi.win_lo];
      C dg = D[doff[0] + idx[0]];
#pragma unroll
      for (int d = 1; d < ND; ++d) dg = cadd(dg, D[doff[d] + idx[d]]);
      C k = cmul(dg, uc);
      for (int t = 0; t < nt; ++t) {
        const TermDesc& td = st[t];
        T wx = (T)1, wy = (T)1;
        for (int i = 0; i < td.n_act; ++i) {
          const int d = td.dim[i];
          const T wv = W[td.wtab[i] + idx[d]];
          if (d < NM) wx *= wv; else wy *= wv;
        }
        const T w = wx * wy;
        const int src = (w != (T)0) ? p + td.deltaR : p;
        k = cfma(sc[t], cscale(win[src - wi.win_lo], w), k);
        if (td.side == SIDE_S && sd.has_sep) {
          const int sx = (wx != (T)0) ? kx + td.deltaGx : kx;
          const int sy = (wy != (T)0) ? ly + td.deltaGy : ly;
          k = cfma(sc[t], cmul(cscale(gxs[sx], wx), cscale(gys[sy], wy)), k);
        }
      }
      combine(sd.off_r + p, uc, k);
    }
  }

  // ---- separable part: G_x (left operator + C) and G_y (right operator - C) --------
  if (sd.has_sep && wi.do_sep) {
    const C Cc = cmk<C>(sd.c_re, sd.c_im);
    const int ng = sd.n_g;
    for (int i = tid; i < 2 * ng; i += blockDim.x) {
      const int side = i < ng ? SIDE_X : SIDE_Y;
      const int g = side == SIDE_X ? i : i - ng;
      const int d0 = side == SIDE_X ? 0 : NM;
      int idx[ND];
      {
        int r = g;
#pragma unroll
        for (int d = NM - 1; d >= 0; --d) { idx[d0 + d] = r % Md[d]; r /= Md[d]; }
      }
      const C* gs = side == SIDE_X ? gxs : gys;
      const C uc = gs[g];
      C dg = side == SIDE_X ? Cc : cmk<C>(-sd.c_re, -sd.c_im);
#pragma unroll
      for (int d = 0; d < NM; ++d) dg = cadd(dg, D[doff[d0 + d] + idx[d0 + d]]);
      C k = cmul(dg, uc);
      for (int t = 0; t < nt; ++t) {
        const TermDesc& td = st[t];
        if (td.side != side) continue;
        T w = (T)1;
        for (int j = 0; j < td.n_act; ++j) w *= W[td.wtab[j] + idx[td.dim[j]]];
        const int delta = side == SIDE_X ? td.deltaGx : td.deltaGy;
        const int src = (w != (T)0) ? g + delta : g;
        k = cfma(sc[t], cscale(gs[src], w), k);
      }
      combine((side == SIDE_X ? sd.off_gx : sd.off_gy) + g, uc, k);
    }
  }

  // ---- step bookkeeping: the last CTA of stage 4 advances the step counter ----------
  if (stage == 4) {
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      const unsigned int t = atomicAdd(A.ticket, 1u);
      if (t == gridDim.x - 1) {
        *A.ticket = 0u;
        *A.counter = *(volatile long long*)A.counter + 1;
        __threadfence();
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Fused RK4 stage, single-mode fast path (the batched workloads of the paper's oscillator
// family).  One CTA holds one whole system: R (M x M), G_x, G_y, the diagonal tables and the
// weight tables of its few stencil terms, all in shared memory.  The term program (counts,
// shifts, table offsets) is precompiled on the host into one M1Sys record per system, read
// with one coalesced load, so a CTA has exactly two barriers.  Per point:
//   k(k,l) = (D_x[k] + D_y[l]) u[k,l] + sum_X c W[k] u[k+s,l] + sum_Y c W[l] u[k,l+s]
//          + sum_S c Wx[k] Wy[l] (u[k+sx,l+sy] + G_x[k+sx] G_y[l+sy]).
// Out-of-grid sources have zero weight; their (clamped) address stays inside the tile.
// ---------------------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T dev_exp(T x);
template <> __device__ __forceinline__ double dev_exp<double>(double x) { return exp(x); }
template <> __device__ __forceinline__ float dev_exp<float>(float x) { return expf(x); }

// Envelope value in the state's precision (FP32 envelopes are accurate to ~1e-7 relative,
// far inside the FP32 path's tolerance; FP64 states evaluate in FP64).
template <typename T>
__device__ double2 chan_value_t(const ChanDesc& c, const double* p, double t) {
  p += c.par_off;
  if (c.kind == 1) {
    const T d = (T)(t - p[2]);
    const T e = dev_exp<T>(-(d * d) / ((T)2 * (T)p[3] * (T)p[3]));
    return make_double2(p[0] * (double)e, p[1] * (double)e);
  }
  return chan_value(c, p - c.par_off, t);
}

template <typename T, int MX, int MY, int MS>
__global__ void __launch_bounds__(BQ_BLOCK) k_stage_m1(const StageArgs A, const M1Sys* __restrict__ m1) {
  using C = typename C2T<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ M1Sys s;
  __shared__ C coef[3 * BQ_M1_MAXT];
  __shared__ double s_tau;
  const int tid = threadIdx.x;
  {
    const int* src = reinterpret_cast<const int*>(m1 + blockIdx.x);
    int* dst = reinterpret_cast<int*>(&s);
    for (int i = tid; i < (int)(sizeof(M1Sys) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    if (tid == 0) s_tau = A.tau_base[0] + (double)(*(volatile long long*)A.counter) * A.dt;
  }
  __syncthreads();
  const int M = s.M, nX = s.nX, nY = s.nY, nS = s.nS;
  const int has_r = s.has_r, has_sep = s.has_sep;
  const int nr = has_r ? M * M : 0;
  // shared layout: u[M*M] | gx[M] | gy[M] | dx[M] | dy[M] | wX[nX*M] wY[nY*M] wSx[nS*M] wSy[nS*M] (real)
  C* u = reinterpret_cast<C*>(smem_raw);
  C* gx = u + nr;
  C* gy = gx + M;
  C* dx = gy + M;
  C* dy = dx + M;
  T* wt = reinterpret_cast<T*>(dy + M);
  T* wX = wt;
  T* wY = wX + nX * M;
  T* wSx = wY + nY * M;
  T* wSy = wSx + nS * M;
  // term coefficients at this stage's time (one thread per term)
  {
    const int nt = nX + nY + nS;
    if (tid < nt) {
      const int t = tid < nX ? s.tX[tid] : (tid < nX + nY ? s.tY[tid - nX] : s.tS[tid - nX - nY]);
      const TermDesc& td = A.terms[s.term_off + t];
      double2 c = make_double2(td.c_re, td.c_im);
      if (td.ch >= 0) {
        const ChanDesc cd = A.chans[td.ch];
        const double tau = (cd.kind == 2) ? s_tau + 0.5 * A.dt : s_tau + stage_c(A.stage) * A.dt;
        double2 e = chan_value_t<T>(cd, A.chpar, A.reverse ? A.horizon - tau : tau);
        if (td.conj) e.y = -e.y;
        c = make_double2(c.x * e.x - c.y * e.y, c.x * e.y + c.y * e.x);
      }
      coef[tid] = cmk<C>(c.x, c.y);
    }
  }
  const C* uin = reinterpret_cast<const C*>(A.u_in);
  if (has_r) {
    const C* src = uin + s.off_r;
    for (int i = tid; i < nr; i += blockDim.x) u[i] = src[i];
  }
  if (has_sep)
    for (int i = tid; i < M; i += blockDim.x) {
      gx[i] = uin[s.off_gx + i];
      gy[i] = uin[s.off_gy + i];
    }
  {
    const C* Dg = reinterpret_cast<const C*>(A.diag) + s.diag_off;
    const T* W = reinterpret_cast<const T*>(A.wtab);
    for (int i = tid; i < M; i += blockDim.x) {
      dx[i] = Dg[i];
      dy[i] = Dg[M + i];
#pragma unroll
      for (int j = 0; j < MX; ++j) if (j < nX) wX[j * M + i] = s.wX[j] >= 0 ? W[s.wX[j] + i] : (T)1;
#pragma unroll
      for (int j = 0; j < MY; ++j) if (j < nY) wY[j * M + i] = s.wY[j] >= 0 ? W[s.wY[j] + i] : (T)1;
#pragma unroll
      for (int j = 0; j < MS; ++j)
        if (j < nS) {
          wSx[j * M + i] = s.wSx[j] >= 0 ? W[s.wSx[j] + i] : (T)1;
          wSy[j * M + i] = s.wSy[j] >= 0 ? W[s.wSy[j] + i] : (T)1;
        }
    }
  }
  __syncthreads();

  C cX[MX], cY[MY], cS[MS];
  int shX[MX], shY[MY], shSx[MS], shSy[MS];
#pragma unroll
  for (int j = 0; j < MX; ++j) { cX[j] = coef[min(j, 3 * BQ_M1_MAXT - 1)]; shX[j] = s.sX[j]; }
#pragma unroll
  for (int j = 0; j < MY; ++j) { cY[j] = coef[min(nX + j, 3 * BQ_M1_MAXT - 1)]; shY[j] = s.sY[j]; }
#pragma unroll
  for (int j = 0; j < MS; ++j) { cS[j] = coef[min(nX + nY + j, 3 * BQ_M1_MAXT - 1)]; shSx[j] = s.sSx[j]; shSy[j] = s.sSy[j]; }

  C* uout = reinterpret_cast<C*>(A.u_out);
  C* y = reinterpret_cast<C*>(A.y);
  C* acc = reinterpret_cast<C*>(A.acc);
  C* comp = reinterpret_cast<C*>(A.comp);
  const T dt = (T)A.dt;
  const int stage = A.stage;
  auto combine = [&](int64_t gi, C uc, C kv) {
    if (stage == 1) {
      uout[gi] = caxpy(dt * (T)0.5, kv, uc);
      acc[gi] = kv;
    } else if (stage == 4) {
      const C yv = y[gi];
      const C sm = cadd(acc[gi], kv);
      const C cv = comp[gi];
      C d, t, c2;
      d.x = dt * (T)(1.0 / 6.0) * sm.x - cv.x;
      d.y = dt * (T)(1.0 / 6.0) * sm.y - cv.y;
      t.x = yv.x + d.x;
      t.y = yv.y + d.y;
      c2.x = (t.x - yv.x) - d.x;
      c2.y = (t.y - yv.y) - d.y;
      y[gi] = t;
      comp[gi] = c2;
    } else {
      const C yv = y[gi];
      uout[gi] = caxpy(stage == 2 ? dt * (T)0.5 : dt, kv, yv);
      acc[gi] = caxpy((T)2, kv, acc[gi]);
    }
  };

  if (has_r) {
    const float invM = 1.0f / (float)M;
    for (int p = tid; p < nr; p += blockDim.x) {
      const int kx = (int)(((float)p + 0.5f) * invM);
      const int ly = p - kx * M;
      const C uc = u[p];
      C kv = cmul(cadd(dx[kx], dy[ly]), uc);
#pragma unroll
      for (int j = 0; j < MX; ++j)
        if (j < nX) {
          const int r = min(max(kx + shX[j], 0), M - 1);
          kv = cfma(cX[j], cscale(u[r * M + ly], wX[j * M + kx]), kv);
        }
#pragma unroll
      for (int j = 0; j < MY; ++j)
        if (j < nY) {
          const int c = min(max(ly + shY[j], 0), M - 1);
          kv = cfma(cY[j], cscale(u[kx * M + c], wY[j * M + ly]), kv);
        }
#pragma unroll
      for (int j = 0; j < MS; ++j)
        if (j < nS) {
          const int r = min(max(kx + shSx[j], 0), M - 1);
          const int c = min(max(ly + shSy[j], 0), M - 1);
          C v = u[r * M + c];
          if (has_sep) v = cadd(v, cmul(gx[r], gy[c]));
          kv = cfma(cS[j], cscale(v, wSx[j * M + kx] * wSy[j * M + ly]), kv);
        }
      combine(s.off_r + p, uc, kv);
    }
  }
  if (has_sep) {
    for (int i = tid; i < 2 * M; i += blockDim.x) {
      const bool isx = i < M;
      const int g = isx ? i : i - M;
      const C* gs = isx ? gx : gy;
      C dg = isx ? cadd(dx[g], cmk<C>(s.c_re, s.c_im)) : cadd(dy[g], cmk<C>(-s.c_re, -s.c_im));
      C kv = cmul(dg, gs[g]);
      if (isx) {
#pragma unroll
        for (int j = 0; j < MX; ++j)
          if (j < nX) kv = cfma(cX[j], cscale(gs[min(max(g + shX[j], 0), M - 1)], wX[j * M + g]), kv);
      } else {
#pragma unroll
        for (int j = 0; j < MY; ++j)
          if (j < nY) kv = cfma(cY[j], cscale(gs[min(max(g + shY[j], 0), M - 1)], wY[j * M + g]), kv);
      }
      combine((isx ? s.off_gx : s.off_gy) + g, gs[g], kv);
    }
  }
  if (stage == 4) {
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      const unsigned int t = atomicAdd(A.ticket, 1u);
      if (t == gridDim.x - 1) {
        *A.ticket = 0u;
        *A.counter = *(volatile long long*)A.counter + 1;
        __threadfence();
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Batched persistent solve (single mode): one launch integrates every system for n_steps.
// Each CTA takes systems from an atomic queue (largest first), keeps the two RK4 stage
// buffers [R | G_x | G_y] in shared memory and the state y, the stage sum and the
// rounding compensation of the points it owns in registers, and runs all steps with one
// barrier per stage.  Drive coefficients of the next stage are evaluated by a few threads
// while the others compute.  There is no inter-CTA waiting of any kind.
// ---------------------------------------------------------------------------------------
template <typename T, int BLK, int PPT, int MX, int MY, int MS>
__global__ void __launch_bounds__(BLK, 2) k_solve_m1(const SolveArgs A) {
  using C = typename C2T<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ M1Sys s;
  __shared__ C coef[2][3 * BQ_M1_MAXT];
  __shared__ int s_next;
  const int tid = threadIdx.x;
  C* y_g = reinterpret_cast<C*>(A.y);
  C* comp_g = reinterpret_cast<C*>(A.comp);

  for (;;) {
    if (tid == 0) s_next = (int)atomicAdd(A.queue, 1u);
    __syncthreads();
    const int qi = s_next;
    if (qi >= A.n_sys) return;
    {
      const int* src = reinterpret_cast<const int*>(A.m1 + A.order[qi]);
      int* dst = reinterpret_cast<int*>(&s);
      for (int i = tid; i < (int)(sizeof(M1Sys) / sizeof(int)); i += BLK) dst[i] = src[i];
    }
    __syncthreads();
    const int M = s.M, nX = s.nX, nY = s.nY, nS = s.nS;
    const int has_r = s.has_r, has_sep = s.has_sep;
    const int nr = has_r ? M * M : 0;
    const int ntot = nr + (has_sep ? 2 * M : 0);
    // shared: B0[ntot] | B1[ntot] | dx[M] | dy[M] | weights (real)
    C* B0 = reinterpret_cast<C*>(smem_raw);
    C* B1 = B0 + ntot;
    C* dx = B1 + ntot;
    C* dy = dx + M;
    T* wX = reinterpret_cast<T*>(dy + M);
    T* wY = wX + nX * M;
    T* wSx = wY + nY * M;
    T* wSy = wSx + nS * M;
    const int nt = nX + nY + nS;
    auto eval_coef = [&](int buf, int64_t step, int stage) {
      if (tid < nt) {
        const int t = tid < nX ? s.tX[tid] : (tid < nX + nY ? s.tY[tid - nX] : s.tS[tid - nX - nY]);
        const TermDesc& td = A.terms[s.term_off + t];
        double2 c = make_double2(td.c_re, td.c_im);
        if (td.ch >= 0) {
          const ChanDesc cd = A.chans[td.ch];
          const double ts = A.tau0 + (double)step * A.dt;
          const double tau = (cd.kind == 2) ? ts + 0.5 * A.dt : ts + stage_c(stage) * A.dt;
          double2 e = chan_value_t<T>(cd, A.chpar, A.reverse ? A.horizon - tau : tau);
          if (td.conj) e.y = -e.y;
          c = make_double2(c.x * e.x - c.y * e.y, c.x * e.y + c.y * e.x);
        }
        coef[buf][tid] = cmk<C>(c.x, c.y);
      }
    };
    // global index of element e of [R | G_x | G_y]
    auto gidx = [&](int e) -> int64_t {
      return e < nr ? s.off_r + e : (e < nr + M ? s.off_gx + (e - nr) : s.off_gy + (e - nr - M));
    };
    C yv[PPT], av[PPT], cv[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int e = tid + j * BLK;
      if (e < ntot) {
        const int64_t g = gidx(e);
        yv[j] = y_g[g];
        cv[j] = comp_g[g];
        B0[e] = yv[j];
      }
    }
    {
      const C* Dg = reinterpret_cast<const C*>(A.diag) + s.diag_off;
      const T* W = reinterpret_cast<const T*>(A.wtab);
      for (int i = tid; i < M; i += BLK) {
        dx[i] = Dg[i];
        dy[i] = Dg[M + i];
#pragma unroll
        for (int j = 0; j < MX; ++j) if (j < nX) wX[j * M + i] = s.wX[j] >= 0 ? W[s.wX[j] + i] : (T)1;
#pragma unroll
        for (int j = 0; j < MY; ++j) if (j < nY) wY[j * M + i] = s.wY[j] >= 0 ? W[s.wY[j] + i] : (T)1;
#pragma unroll
        for (int j = 0; j < MS; ++j)
          if (j < nS) {
            wSx[j * M + i] = s.wSx[j] >= 0 ? W[s.wSx[j] + i] : (T)1;
            wSy[j * M + i] = s.wSy[j] >= 0 ? W[s.wSy[j] + i] : (T)1;
          }
      }
    }
    eval_coef(0, 0, 1);
    int shX[MX], shY[MY], shSx[MS], shSy[MS];
#pragma unroll
    for (int j = 0; j < MX; ++j) shX[j] = s.sX[j];
#pragma unroll
    for (int j = 0; j < MY; ++j) shY[j] = s.sY[j];
#pragma unroll
    for (int j = 0; j < MS; ++j) { shSx[j] = s.sSx[j]; shSy[j] = s.sSy[j]; }
    const C Cc = cmk<C>(s.c_re, s.c_im);
    const T dt = (T)A.dt;
    const float invM = 1.0f / (float)M;
    __syncthreads();

    int buf = 0;
    for (int64_t step = 0; step < A.n_steps; ++step) {
#pragma unroll 1
      for (int stage = 1; stage <= 4; ++stage) {
        const C* uin = (stage & 1) ? B0 : B1;  // stages 1, 3 read B0; 2, 4 read B1
        C* uout = (stage & 1) ? B1 : B0;
        C cX[MX], cY[MY], cS[MS];
#pragma unroll
        for (int j = 0; j < MX; ++j) cX[j] = coef[buf][min(j, 3 * BQ_M1_MAXT - 1)];
#pragma unroll
        for (int j = 0; j < MY; ++j) cY[j] = coef[buf][min(nX + j, 3 * BQ_M1_MAXT - 1)];
#pragma unroll
        for (int j = 0; j < MS; ++j) cS[j] = coef[buf][min(nX + nY + j, 3 * BQ_M1_MAXT - 1)];
        const C* gxi = uin + nr;
        const C* gyi = gxi + M;
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
          const int e = tid + j * BLK;
          if (e >= ntot) continue;
          const C uc = uin[e];
          C kv;
          if (e < nr) {
            const int kx = (int)(((float)e + 0.5f) * invM);
            const int ly = e - kx * M;
            kv = cmul(cadd(dx[kx], dy[ly]), uc);
#pragma unroll
            for (int q = 0; q < MX; ++q)
              if (q < nX) kv = cfma(cX[q], cscale(uin[min(max(kx + shX[q], 0), M - 1) * M + ly], wX[q * M + kx]), kv);
#pragma unroll
            for (int q = 0; q < MY; ++q)
              if (q < nY) kv = cfma(cY[q], cscale(uin[kx * M + min(max(ly + shY[q], 0), M - 1)], wY[q * M + ly]), kv);
#pragma unroll
            for (int q = 0; q < MS; ++q)
              if (q < nS) {
                const int r = min(max(kx + shSx[q], 0), M - 1);
                const int c = min(max(ly + shSy[q], 0), M - 1);
                C v = uin[r * M + c];
                if (has_sep) v = cadd(v, cmul(gxi[r], gyi[c]));
                kv = cfma(cS[q], cscale(v, wSx[q * M + kx] * wSy[q * M + ly]), kv);
              }
          } else {
            const bool isx = e < nr + M;
            const int g = isx ? e - nr : e - nr - M;
            const C* gs = isx ? gxi : gyi;
            kv = cmul(isx ? cadd(dx[g], Cc) : cadd(dy[g], cmk<C>(-s.c_re, -s.c_im)), uc);
            if (isx) {
#pragma unroll
              for (int q = 0; q < MX; ++q)
                if (q < nX) kv = cfma(cX[q], cscale(gs[min(max(g + shX[q], 0), M - 1)], wX[q * M + g]), kv);
            } else {
#pragma unroll
              for (int q = 0; q < MY; ++q)
                if (q < nY) kv = cfma(cY[q], cscale(gs[min(max(g + shY[q], 0), M - 1)], wY[q * M + g]), kv);
            }
          }
          // RK4 combine (stage sum + compensated state update, as in the stage kernels)
          if (stage == 1) {
            uout[e] = caxpy(dt * (T)0.5, kv, yv[j]);
            av[j] = kv;
          } else if (stage == 4) {
            const C sm = cadd(av[j], kv);
            C d, t;
            d.x = dt * (T)(1.0 / 6.0) * sm.x - cv[j].x;
            d.y = dt * (T)(1.0 / 6.0) * sm.y - cv[j].y;
            t.x = yv[j].x + d.x;
            t.y = yv[j].y + d.y;
            cv[j].x = (t.x - yv[j].x) - d.x;
            cv[j].y = (t.y - yv[j].y) - d.y;
            yv[j] = t;
            uout[e] = t;
          } else {
            uout[e] = caxpy(stage == 2 ? dt * (T)0.5 : dt, kv, yv[j]);
            av[j] = caxpy((T)2, kv, av[j]);
          }
        }
        // coefficients of the next stage (stage 4 -> stage 1 of the next step)
        const int nstage = stage == 4 ? 1 : stage + 1;
        eval_coef(buf ^ 1, stage == 4 ? step + 1 : step, nstage);
        buf ^= 1;
        __syncthreads();
      }
    }
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int e = tid + j * BLK;
      if (e < ntot) {
        const int64_t g = gidx(e);
        y_g[g] = yv[j];
        comp_g[g] = cv[j];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Observables: one warp per evaluation group, lanes over (initial condition, entry) pairs.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void k_eval(const SysDesc* __restrict__ sys, const EvalGroup* __restrict__ groups,
                       const EvalEntry* __restrict__ entries, const void* ystate, double2* out,
                       int n_groups) {
  using C = typename C2T<T>::type;
  const C* y = reinterpret_cast<const C*>(ystate);
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n_groups) return;
  const EvalGroup g = groups[warp];
  double re = 0.0, im = 0.0;
  const int total = g.n_sys * g.n_e;
  for (int i = lane; i < total; i += 32) {
    const int s = i / g.n_e;
    const int e = i - s * g.n_e;
    const SysDesc& sd = sys[g.sys_off + s];
    const EvalEntry en = entries[g.e_off + e];
    double vr = 0.0, vi = 0.0;
    if (sd.has_sep) {
      const C a = y[sd.off_gx + en.kx];
      const C b = y[sd.off_gy + en.ly];
      vr += (double)a.x * (double)b.x - (double)a.y * (double)b.y;
      vi += (double)a.x * (double)b.y + (double)a.y * (double)b.x;
    }
    if (sd.has_r) {
      const C r = y[sd.off_r + (int64_t)en.kx * sd.n_g + en.ly];
      vr += (double)r.x;
      vi += (double)r.y;
    }
    // w * f * v
    const double fr = sd.w_re * en.f_re - sd.w_im * en.f_im;
    const double fi = sd.w_re * en.f_im + sd.w_im * en.f_re;
    re += fr * vr - fi * vi;
    im += fr * vi + fi * vr;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
  }
  if (lane == 0) out[warp] = make_double2(re, im);
}

// Observables for groups with few (initial condition, entry) pairs: one thread per group.
template <typename T>
__global__ void k_eval_small(const SysDesc* __restrict__ sys, const EvalGroup* __restrict__ groups,
                             const EvalEntry* __restrict__ entries, const void* ystate, double2* out, int n_groups) {
  using C = typename C2T<T>::type;
  const C* y = reinterpret_cast<const C*>(ystate);
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= n_groups) return;
  const EvalGroup g = groups[gi];
  double re = 0.0, im = 0.0;
  for (int s = 0; s < g.n_sys; ++s) {
    const SysDesc& sd = sys[g.sys_off + s];
    const double wr = sd.w_re, wim = sd.w_im;
    const int sep = sd.has_sep, hr = sd.has_r, ng = sd.n_g;
    const int64_t ox = sd.off_gx, oy = sd.off_gy, orr = sd.off_r;
    for (int e = 0; e < g.n_e; ++e) {
      const EvalEntry en = entries[g.e_off + e];
      double vr = 0.0, vi = 0.0;
      if (sep) {
        const C a = y[ox + en.kx];
        const C b = y[oy + en.ly];
        vr += (double)a.x * (double)b.x - (double)a.y * (double)b.y;
        vi += (double)a.x * (double)b.y + (double)a.y * (double)b.x;
      }
      if (hr) {
        const C r = y[orr + (int64_t)en.kx * ng + en.ly];
        vr += (double)r.x;
        vi += (double)r.y;
      }
      const double fr = wr * en.f_re - wim * en.f_im;
      const double fi = wr * en.f_im + wim * en.f_re;
      re += fr * vr - fi * vi;
      im += fr * vi + fi * vr;
    }
  }
  out[gi] = make_double2(re, im);
}

// Initial state: y[off] = value for a list of (offset, value) pairs (the rest is zeroed).
template <typename T>
__global__ void k_scatter(const InitEntry* __restrict__ ent, int n, void* ystate) {
  using C = typename C2T<T>::type;
  C* y = reinterpret_cast<C*>(ystate);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[ent[i].off] = cmk<C>(ent[i].re, ent[i].im);
}

// ---------------------------------------------------------------------------------------
// Fixed RK4 scratch for callers that cannot allocate device memory.
//
// bq_step_fixed_scratch() takes the two stage buffers and the RK4 accumulator from this
// file-scope array instead of from the state's pool.  Every GPU that loads the library
// holds it until the process exits.  Host code must not use the symbol's name as an
// address: fixed_scratch() looks the device address up once per device.
// ---------------------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_fixed_scratch[3 * BQ_FIXED_SCRATCH_BYTES];

cudaError_t fixed_scratch(void** ptr) {
  static std::mutex mu;
  static void* cache[256] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!cache[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fixed_scratch);
    if (e != cudaSuccess) return e;
    cache[dev] = p;
  }
  *ptr = cache[dev];
  return cudaSuccess;
}

// ---------------------------------------------------------------------------------------
// Host-side launchers.
// ---------------------------------------------------------------------------------------
template <typename T, int NM>
static cudaError_t launch_stage_t(const StageArgs& a, int n_work, int smem_bytes, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_stage<T, NM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         BQ_MAX_DYN_SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_stage<T, NM><<<n_work, BQ_BLOCK, smem_bytes, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int MX, int MY, int MS>
static cudaError_t launch_stage_m1_t(const StageArgs& a, const M1Sys* m1, int n_work, int smem_bytes, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_stage_m1<T, MX, MY, MS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         BQ_MAX_DYN_SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_stage_m1<T, MX, MY, MS><<<n_work, BQ_BLOCK, smem_bytes, s>>>(a, m1);
  return cudaGetLastError();
}

cudaError_t launch_stage_m1(const StageArgs& a, const M1Sys* m1, int variant, int dtype, int n_work, int smem_bytes,
                            cudaStream_t s) {
  // variant 0: at most 2 terms per side; variant 1: at most BQ_M1_MAXT
  if (dtype == 0)
    return variant == 0 ? launch_stage_m1_t<double, 2, 2, 2>(a, m1, n_work, smem_bytes, s)
                        : launch_stage_m1_t<double, BQ_M1_MAXT, BQ_M1_MAXT, BQ_M1_MAXT>(a, m1, n_work, smem_bytes, s);
  return variant == 0 ? launch_stage_m1_t<float, 2, 2, 2>(a, m1, n_work, smem_bytes, s)
                      : launch_stage_m1_t<float, BQ_M1_MAXT, BQ_M1_MAXT, BQ_M1_MAXT>(a, m1, n_work, smem_bytes, s);
}

template <typename T, int BLK, int PPT>
static cudaError_t launch_solve_t(const SolveArgs& a, int smem_bytes, cudaStream_t s, int* grid_out) {
  auto kern = k_solve_m1<T, BLK, PPT, 2, 2, 2>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, BQ_MAX_DYN_SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLK, smem_bytes);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::min(a.n_sys, per_sm * nsm);
  *grid_out = grid;
  kern<<<grid, BLK, smem_bytes, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_solve_m1(const SolveArgs& a, int dtype, int capacity_class, int smem_bytes, cudaStream_t s,
                            int* grid_out) {
  // capacity: FP32 256 threads x 7 points = 1792, FP64 448 threads x 4 points = 1792 points per system
  if (capacity_class != 0) return cudaErrorInvalidValue;
  return dtype == 0 ? launch_solve_t<double, 448, 4>(a, smem_bytes, s, grid_out)
                    : launch_solve_t<float, 256, 7>(a, smem_bytes, s, grid_out);
}

cudaError_t launch_stage(const StageArgs& a, int dtype, int nm, int n_work, int smem_bytes, cudaStream_t s) {
  if (dtype == 0) {
    switch (nm) {
      case 1: return launch_stage_t<double, 1>(a, n_work, smem_bytes, s);
      case 2: return launch_stage_t<double, 2>(a, n_work, smem_bytes, s);
      case 3: return launch_stage_t<double, 3>(a, n_work, smem_bytes, s);
    }
  } else {
    switch (nm) {
      case 1: return launch_stage_t<float, 1>(a, n_work, smem_bytes, s);
      case 2: return launch_stage_t<float, 2>(a, n_work, smem_bytes, s);
      case 3: return launch_stage_t<float, 3>(a, n_work, smem_bytes, s);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_eval(const SysDesc* sys, const EvalGroup* groups, const EvalEntry* entries, const void* y,
                        double2* out, int n_groups, int dtype, int small, cudaStream_t s) {
  if (n_groups <= 0) return cudaSuccess;
  const int threads = 256;
  if (small) {
    const int blocks = (n_groups + threads - 1) / threads;
    if (dtype == 0)
      k_eval_small<double><<<blocks, threads, 0, s>>>(sys, groups, entries, y, out, n_groups);
    else
      k_eval_small<float><<<blocks, threads, 0, s>>>(sys, groups, entries, y, out, n_groups);
    return cudaGetLastError();
  }
  const int blocks = (n_groups * 32 + threads - 1) / threads;
  if (dtype == 0)
    k_eval<double><<<blocks, threads, 0, s>>>(sys, groups, entries, y, out, n_groups);
  else
    k_eval<float><<<blocks, threads, 0, s>>>(sys, groups, entries, y, out, n_groups);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const InitEntry* ent, int n, void* y, int dtype, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  const int blocks = (n + threads - 1) / threads;
  if (dtype == 0)
    k_scatter<double><<<blocks, threads, 0, s>>>(ent, n, y);
  else
    k_scatter<float><<<blocks, threads, 0, s>>>(ent, n, y);
  return cudaGetLastError();
}

}  // namespace bq
