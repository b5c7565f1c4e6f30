// Internal data structures shared by the host compiler and the CUDA kernels.
// All structs are plain-old-data with identical layout on host and device; they are
// written into the caller's device pool by bq_map() and read by the kernels.
#pragma once

#include <stdint.h>
#include <vector_types.h>

#define BQ_MAXD 8          // max R dimensions = 2 * BQ_MAX_MODES
#define BQ_MAX_TERMS 64    // max general (non-folded) stencil terms per problem
#define BQ_BLOCK 128       // threads per CTA of the stage kernels

namespace bq {

enum Side : int { SIDE_X = 0, SIDE_Y = 1, SIDE_S = 2 };

// One general stencil term of the coupled system (Eqs. 9a-c): a monomial x^a d^b in
// each of its active dimensions (x-dims 0..nm-1, y-dims nm..2nm-1 of R).
//  * SIDE_X: left multiplication of A by an operator  -> acts on G_x and on R's x-dims;
//  * SIDE_Y: right multiplication                     -> acts on G_y and on R's y-dims;
//  * SIDE_S: sandwich L^dag A L                       -> acts on R (x- and y-dims at once)
//            and is the source S(G_x G_y) of Eq. 9c / 303c.
// The value added at point k is coef(t) * prod_i W_i[k_dim_i] * u[k + delta], where
// W_i is a weight table (zero where the source index leaves the grid).
struct TermDesc {
  double c_re, c_im;   // static part of the coefficient (rate, param, basis factors folded in)
  int ch;              // channel index into the state's channel table, -1 = static
  int conj;            // multiply by conj(channel) instead of channel
  int side;            // Side
  int n_act;           // number of active dimensions
  int deltaR;          // linear source offset in R
  int deltaGx;         // linear source offset in G_x (SIDE_X, SIDE_S x-part)
  int deltaGy;         // linear source offset in G_y (SIDE_Y, SIDE_S y-part)
  int param;           // gradient parameter index or -1 (coefficient = theta * c)
  int8_t dim[BQ_MAXD];
  int8_t diagp1;       // 0: everywhere; j + 1: only where the x and y indices of mode j agree
  int8_t pad8;
  int wtab[BQ_MAXD];   // element offsets of the weight tables (length M_dim each)
  // gradient metadata
  double cb_re, cb_im; // coefficient with the parameter value set to 1
  int8_t sh[BQ_MAXD];  // source shift (b - a) per active dimension
  int8_t pad8b[2];
  int gslot_param;     // gradient slot of d/dtheta (absolute, -1: none)
  int gslot_pwc;       // gradient slot of Re(segment 0) of a piecewise-constant channel (-1: none)
};

// Drive envelope.
struct ChanDesc {
  int kind;
  int n_par;
  int par_off;  // into the channel parameter pool (double)
  int pad;
};

// One system = one separable initial condition of one problem (or one direct state).
struct SysDesc {
  int prob;             // problem index in the batch
  int nm;               // number of modes
  int M[BQ_MAXD / 2];   // grid per mode
  int has_sep;          // G_x, G_y present (mapped method)
  int has_r;            // R present
  int n_g;              // elements of G_x (= of G_y) = prod M
  int n_r;              // elements of R = n_g^2
  int term_off, n_terms;
  int diag_off;         // complex element offset of 2*nm diagonal tables (length M_d each)
  int halo_lo, halo_hi; // max negative / positive linear offset of any R term
  int p_flat, q_flat;   // initial condition indices (flattened)
  int stR[BQ_MAXD];     // element strides of R (x-dims outer, y-dims inner)
  int stG[BQ_MAXD / 2]; // element strides of G_x / G_y
  int dc_off;           // offset of d C / d theta_p (complex, one per parameter) in the gradient tables
  int64_t off_gx, off_gy, off_r;  // complex element offsets into the state arrays
  double c_re, c_im;    // separation constant C (Eq. 304)
  double w_re, w_im;    // weight g_{p,q}(0) of the initial condition
  int n_params;         // parameters of the problem
  int grad_off;         // gradient slot of the problem's first parameter
  int r_diag;           // R stored only at k = l (n_r = n_g entries, index = flat k)
  int n_sterms;         // sandwich terms of the system's problem (adjoint source reductions)
  int cw_elems;         // complex elements of the tiled kernel's coefficient x weight tables
};

// A CTA's share of one stage: a tile of R points of one system (plus G_x, G_y if sep).
struct WorkItem {
  int sys;
  int start, len;       // R tile [start, start + len)
  int sep_lo, sep_hi;   // G points [sep_lo, sep_hi) of [G_x | G_y] (2 n_g) this CTA updates
  int win_lo, win_hi;   // R window staged in shared memory
  int smem_elems;       // complex elements of shared memory this item needs
  int gread;            // 1: no R window (the halo does not fit); sources are read from global memory
};

// Evaluation: out[g] = sum_{IC of problem} w_IC * sum_{e in group} f_e * G_IC(k_e, l_e)
// where G_IC(k, l) = gx[k] gy[l] + R[k, l] in storage basis.
struct EvalGroup {
  int prob;
  int e_off, n_e;       // entries
  int sys_off, n_sys;   // systems (ICs) of the problem (contiguous)
  int pad[3];
};
struct EvalEntry {
  int kx, ly;           // flat x-index, flat y-index
  int pad[2];
  double f_re, f_im;    // factor
};

// Single-mode fast path: one record per system with the term program precompiled on the
// host (term counts per side, source shifts, weight-table offsets, term indices).
#define BQ_M1_MAXT 4
struct M1Sys {
  int M, nX, nY, nS;
  int has_sep, has_r, term_off, diag_off;
  int sX[BQ_M1_MAXT], sY[BQ_M1_MAXT], sSx[BQ_M1_MAXT], sSy[BQ_M1_MAXT];
  int wX[BQ_M1_MAXT], wY[BQ_M1_MAXT], wSx[BQ_M1_MAXT], wSy[BQ_M1_MAXT];  // -1: weight 1
  int tX[BQ_M1_MAXT], tY[BQ_M1_MAXT], tS[BQ_M1_MAXT];
  int sdiag;  // bit q: sandwich term q acts only where k = l (secular projector)
  int pad[3];
  int64_t off_gx, off_gy, off_r;
  int64_t pad64;
  double c_re, c_im;
};

struct StageArgs {
  const SysDesc* sys;
  const TermDesc* terms;
  const ChanDesc* chans;
  const double* chpar;
  const void* wtab;     // weight tables (real type of the state)
  const void* diag;     // diagonal tables (complex of the state type)
  const WorkItem* work;
  const void* u_in;     // stage input (y for stage 1)
  void* u_out;          // next stage input (stages 1-3)
  void* y;              // state (read stages 2-3, written stage 4)
  void* acc;            // RK4 stage sum k1 + 2 k2 + 2 k3 (scratch)
  void* comp;           // compensation of the state update (part of the state, starts at 0)
  void* rec;            // if non-null: the stage input of every point is also written here
  const double* tau_base;      // device: tau at counter = 0
  long long* counter;          // device: completed steps since tau_base
  unsigned int* ticket;        // device: stage-4 completion ticket
  double dt;
  double horizon;
  int reverse;
  int stage;            // 1..4
  int lanes;            // lanes per point of the tiled kernel (1, 2 or 4): the terms are split
                        // across them and the partial sums combined with shuffles
};

// Pipelined single-mode stage kernel (k_stage_pipe): one record per system and one
// parameter block per problem, the block fetched with a 1-D bulk copy (TMA) into shared memory
// together with the system's stage input.
struct __align__(16) PipeRec {
  int blk_off;      // element offset of the system block ([G_x | G_y | R] or [R]) in the state arrays
  int blk_elems;    // element count of the block (multiple of 4)
  int param_off;    // byte offset of the problem's parameter block
  int param_bytes;  // its size (multiple of 16)
  int gy_off, r_off;  // element offsets inside the block (-1: absent); G_x, when present, starts it
  int M;            // grid size of the mode
  int merged;       // 1: merged-stencil path (every shift in {-1, 0, 1}, M <= 64)
  int nb, rb;       // merged path: nb column strips of rb rows (thread t: column t % M, strip t / M)
  float inv_m;      // 1 / M (strip index without an integer division)
  float w32_re, w32_im;  // the weight below rounded to FP32 (the FP32 kernels' observable)
  float c32_re, c32_im;  // C below rounded to FP32 (the FP32 kernels' G items)
  int sys;          // index of the system (records are ordered by size, largest first)
  union {
    struct {
      double c_re, c_im;  // separation constant C of the system (Eq. 304)
      double w_re, w_im;  // weight of the system's initial condition
    } d;                  // FP64 kernels
    struct {              // FP32 kernels: the problem's drive envelope when it is one Gaussian
      float amp_re, amp_im, k;  // amplitude, 1 / (2 sigma^2)
      float c_hi, c_lo;         // centre as an unevaluated FP32 pair
      int gauss;                // 1: the fields above are set
      float e_re, e_im;         // its value at the stage time (set in the kernel's copy)
    } f;
  };
};
// Header of a parameter block (128 B), followed by n_terms PipeCoef records (X, Y, S terms in
// program order), n_ch PipeChan records, dx[M], dy[M] (complex) and the weight tables
// wX[nX][M], wY[nY][M], wSx[nS][M], wSy[nS][M] (real), then n_obs PipeObs records at a 16-B
// boundary, the whole block padded to 16 B.
struct PipeHdr {
  int M, nX, nY, nS, has_sep, has_r, ntot, merged;  // merged: all shifts in {-1,0,1}, nS <= 2, M <= 64
  int sX[BQ_M1_MAXT], sY[BQ_M1_MAXT], sSx[BQ_M1_MAXT], sSy[BQ_M1_MAXT];
  int sdiag;    // bit q: sandwich term q acts only where k = l (secular projector)
  int n_terms;  // nX + nY + nS
  int n_ch;     // drive envelopes behind the time-dependent terms (0..2)
  int obs_off;  // byte offset of the PipeObs records (the problem's Tr(rho0 A) entries)
  int n_obs;    // their count (0..32; 0 also when the kernel does not evaluate the observable)
  int pad2[3];
};
// An entry (k, l, f) of rho0's support in a parameter block, f in the state's precision.
template <typename CT>
struct PipeObs {
  int kx, ly;  // flat indices (this path has one mode)
  CT f;
};
// A drive envelope (bq.h channel kinds) in a parameter block: its first four parameters and,
// for a piecewise-constant envelope, the offset and count of its parameters in the state's
// channel parameter pool (the segment values are read from there).
struct PipeChan {
  double p[4];
  int kind, par_off, n_par;
  float c_lo;  // Gaussian: the centre p[2] - f[3] (the FP32 remainder of the centre)
  float f[4];  // the same in FP32: amplitude (re, im), then 1 / (2 sigma^2) and the centre for a Gaussian
};
// Stage coefficient of one term: c times the value of the block's envelope ch (0 or 1, -1:
// static) at the stage time, or its conjugate (conj = 1).
template <typename CT>
struct PipeCoef {
  CT c;
  int ch, conj;
};
#define BQ_PIPE_THREADS 128  // threads of a pipelined stage CTA
#define BQ_MERGED_MAXM 64    // column-vector builders start at this thread
// complex entries of a row / column coefficient record of the merged path (A0, Am, Ap and two
// per sandwich term), rounded up to an even count so that records are 16-byte aligned pairs
#define BQ_PIPE_RS(MS) ((3 + 2 * (MS) + 1) & ~1)

struct PipeArgs {
  const PipeRec* recs;
  const unsigned char* params;
  const ChanDesc* chans;
  const double* chpar;
  const void* u_in;     // stage input (the state y at stage 1)
  void* u_out;
  void* y;
  void* acc;            // stage sum (scratch)
  void* comp;           // rounding residual of the state (part of the state: true value y - comp)
  unsigned int* ticket;
  long long* counter;
  const double* tau_base;
  unsigned int* error;  // set when a bounded wait gives up
  int n_sys, n_slots;
  int slot_bytes, off_u;    // bytes of a shared-memory slot; offset of the stage input in it
  int zero_off, zero_bytes; // guard band before the stage input .. end of the guard band after it
  int mmax, reverse;        // largest M of the state (coefficient records); reversed-time reading
  int comp_zero;            // stage 1: comp is known to be zero (a freshly loaded state); not read
  int pad;
  double2* obs;             // stage 4 (or null): per system, w sum_e f_e G(k_e, l_e) of the updated state
  double dt, horizon;
};

// Arguments of the batched persistent solve (k_solve_m1).
struct SolveArgs {
  const M1Sys* m1;
  const int* order;        // systems, largest first
  const TermDesc* terms;
  const ChanDesc* chans;
  const double* chpar;
  const void* wtab;
  const void* diag;
  void* y;
  void* comp;
  unsigned int* queue;     // device: next queue position (zeroed before the launch)
  int n_sys;
  int reverse;
  int has_diag;            // some system has a diagonal-restricted (secular) sandwich term
  int pad_sa;
  long long n_steps;
  double dt, tau0, horizon;
};

// Arguments of one adjoint (transposed) RK4 stage, see k_adj_stage.
struct AdjArgs {
  const SysDesc* sys;
  const TermDesc* terms;
  const ChanDesc* chans;
  const double* chpar;
  const void* wtab;
  const void* diag;
  const WorkItem* work;
  const double2* dc;     // d C / d theta per system (SysDesc::dc_off)
  const void* b_in;      // b_i; NULL at stage 4 (then b_4 = dt/6 lam)
  const void* lam;       // cotangent of the state after the step
  void* lacc;            // cotangent of the state before the step (accumulated over stages)
  void* b_out;           // b_{i-1} (stages 4..2)
  const void* u;         // recorded stage input u_i
  const void* srcred;    // transposed-source reductions, srcred_stride complex per system
  double* grad;          // gradient slots
  double tau_step, dt, horizon;
  int reverse, stage, srcred_stride;
  int ng_max;            // largest n_g (G_x / G_y points) over the systems
  int lanes;             // lanes per point (1, 2 or 4), as in StageArgs
};

// Cooperative segment kernels of the gradient (k_coop_fwd, k_coop_bwd): all stages of a
// checkpoint segment in one launch, the dependent phases separated by bounded grid barriers.
struct CoopArgs {
  StageArgs st;           // forward template (stage, u_in, u_out, rec set per phase)
  AdjArgs adj;            // adjoint template (stage, u, b_in, b_out, lam, lacc, tau_step set per phase)
  void* ua;               // forward ping-pong stage inputs
  void* ub;
  char* rec;              // recorded stage inputs of the segment (4 per step), or null
  size_t arr;             // bytes of one state array
  void* ba;               // adjoint b ping-pong buffers
  void* bb;
  void* lam;              // cotangent after the segment's last step (swapped with lacc per step)
  void* lacc;
  double tau0;            // tau at the segment's first step
  int n_steps;
  int n_work;             // work items of a stage
  int n_sys, max_s, src_tiles;  // transposed-source items: n_sys x max_s x 2 src_tiles
  unsigned int* bar;      // grid barrier words: [0] arrivals, [1] generation
  unsigned int* error;    // set (bit 2) when a barrier wait gives up
};

}  // namespace bq
