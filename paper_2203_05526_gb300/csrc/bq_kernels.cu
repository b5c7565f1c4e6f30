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

  auto combine = [&](int64_t gi, C uc, C k) {
    if (stage == 1) {
      uout[gi] = caxpy(dt * (T)0.5, k, uc);
      acc[gi] = caxpy(dt * (T)(1.0 / 6.0), k, uc);
    } else if (stage == 4) {
      y[gi] = caxpy(dt * (T)(1.0 / 6.0), k, acc[gi]);
    } else {
      const C yv = y[gi];
      uout[gi] = caxpy(stage == 2 ? dt * (T)0.5 : dt, k, yv);
      acc[gi] = caxpy(dt * (T)(1.0 / 3.0), k, acc[gi]);
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
                        double2* out, int n_groups, int dtype, cudaStream_t s) {
  if (n_groups <= 0) return cudaSuccess;
  const int threads = 256;
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
