// Explicit Boussinesq natural-convection step (Section 3, Eqs. 2-4) with
// Chorin's projection, on the weights of a plan.
//
// Per step (rho = 1, e_up = last axis):
//   1. v* = v + dt[-(v.grad)v + Pr lap v + Ra Pr (T - T_ref) e_up] inside,
//      v* = 0 on walls (no-slip);
//   2. pressure from the bordered system [Lp 1; 1' 0][p; c] = [rhs; 0] with
//      Lp = Laplacian rows inside / normal-derivative rows on walls and
//      rhs = div(v*)/dt inside, 0 on walls; GMRES(30) right-preconditioned
//      by the multigrid cycle (or BiCGSTAB), started from the previous
//      solutions (p, c) extrapolated in time;
//   3. v = v* - dt grad p inside, 0 on walls;
//   4. T = T + dt[-v.grad T + lap T] inside, with the new v;
//   5. Dirichlet walls T = T_bc; insulated walls T_b = -sum_{i>0} wn_i T_i / wn_0
//      (a wall stencil holds only interior nodes besides its centre).
//
// Every kernel walks the two stencil groups of the plan (blocks of the MON
// group first, then the RBF-FD group), one thread per node.  A BiCGSTAB
// iteration is three kernels; each forms the vector it needs on the fly
// inside its gathers (p = r + beta(p - omega v), s = r - alpha v), applies the
// bordered operator right-preconditioned by its diagonal (Jacobi; the
// Laplacian rows scale as 1/h^2 and the wall rows as 1/h, and the unscaled
// iteration stagnates), and reduces its dot products with a last-block-done
// pattern (block partials in fixed order, no spinning), whose final block also
// updates the scalars and the convergence flag.  Once the flag is set the
// remaining kernels of a launched chunk return at once.
//
// With the multigrid preconditioner (the default) a BiCGSTAB iteration forms
// p, runs a V-cycle p -> p^ = M^-1 p, applies the bordered operator
// v = A p^, forms s, runs s -> s^ = M^-1 s, applies t = A s^, and updates x
// and r: five vector/operator kernels around two V-cycles (amg.cu).  A GMRES
// iteration (the default with the multigrid cycle) runs one V-cycle and one
// operator application (section 2d): on the seeded sets, started from the
// extrapolated guess, it needs about as many iterations as BiCGSTAB, so a
// step takes about a quarter less time.
#include <vector>

#include "amg.cuh"
#include "common.cuh"

struct hsm_stepper_s {
  hsm_plan plan = nullptr;
  hsm_phys phys{};
  int dim = 2;
  int64_t N = 0;
  int slot_d[3] = {0, 0, 0};  // weight slot of d/dx_k in the plan
  int slot_lap = 0;
  double* wp_rbf = nullptr;   // [n][rbf_count] pressure-row weights (lap inside, n.grad on walls)
  double* wn_rbf = nullptr;   // [n][rbf_count] normal-derivative weights (walls only)
  double* minv = nullptr;     // [N+1] inverse diagonal of the bordered operator (1 for the border)
  double* vstar = nullptr;    // [dim][N]
  double* Tn = nullptr;       // [N]
  double* vec = nullptr;      // Krylov vectors, each N+1: r, rhat, p0, p1, v0, v1, s, t, rhs
  double* hist = nullptr;     // [2][N+1]: (p, c) of the last two steps, for the extrapolated initial guess
  double* scal = nullptr;     // KrylovScalars
  double* partial = nullptr;  // [3][blocks][4]
  unsigned* counters = nullptr;
  int blocks_mon = 0, blocks_rbf = 0, threads = 256;
  double c = 0.0;             // Lagrange multiplier of the bordered system (kept on device)
  // CUDA graphs of the step phases, valid for the field pointers they were
  // captured with: head = predictor + Krylov set-up + `head_chunks` chunks of
  // Krylov iterations, chunk = one chunk, tail = correction + temperature
  cudaGraphExec_t g_head = nullptr, g_chunk = nullptr, g_tail = nullptr;
  cudaStream_t cap = nullptr;  // private stream the graphs are captured on
  cudaStream_t body = nullptr; // second capture stream (the conditional loop's body)
  int head_chunks = 0;
  const double *gv = nullptr, *gT = nullptr, *gp = nullptr;
  int last_iters = 0;
  hsm::Amg* amg = nullptr;    // multigrid preconditioner (nullptr: Jacobi)
  // one graph per step with the Krylov iterations in a conditional WHILE
  // node: the loop ends on the device, without a host round trip
  cudaGraphExec_t g_step = nullptr;
  bool g_step_failed = false;  // conditional nodes unavailable: host-driven loop
  unsigned* ctl = nullptr;     // [0] iterations of the current loop, [1] steps recorded, [2] loop cap reached
  int* step_iters = nullptr;   // per step of the current hsm_step call
  int* step_bad = nullptr;     // 1 where a step's solve stopped short of its tolerance
  int step_cap = 0;
  // GMRES (hsm_phys.krylov): basis V [M+1], Z [M], vin, zout, w, each N+1;
  // scalars; dot-product partials and their arrival counter
  bool gmres = false;          // GMRES with the multigrid cycle (else BiCGSTAB)
  double* gm_vec = nullptr;
  double* gm_scal = nullptr;
  double* gm_part = nullptr;
  unsigned* gm_cnt = nullptr;
};

namespace hsm {
namespace {

enum { V_R = 0, V_RHAT, V_P0, V_P1, V_V0, V_V1, V_S, V_T, V_RHS, V_PH, V_SH, V_COUNT };

// Scalars of the Krylov solve (device memory, doubles + ints packed as doubles).
struct KS {
  double rho, alpha, omega, beta;
  double bnorm2, rnorm2, tol2;
  double xN;            // Lagrange multiplier c
  double iter, done, breakdown, max_it, half;
  double cur;           // which p/v buffer holds the current iterate (0 or 1)
};

struct StepArgs {
  // plan groups
  const int32_t* nodes[2];
  const int32_t* idx[2];
  const double* w[2];      // plan weights [nops][width][count]
  const float* w32[2];     // their FP32 copies (FP32 operator applications), or nullptr
  const double* wp[2];     // pressure weights of the group ([width][count])
  const double* wn[2];     // wall normal-derivative weights (rbf group only)
  int64_t count[2];
  int width[2];
  int64_t bm;              // blocks of the MON group
  int slot_d[3];
  int slot_lap;
  int dim;
  int64_t N;
  // physics
  double Ra, Pr, dt, T_ref;
  const uint8_t* bc;
  const double* T_bc;
  // fields
  double* v;
  double* T;
  double* p;
  double* vstar;
  double* Tn;
  double* vec;
  double* hist;            // [2][N+1] (p, c) of the previous two steps
  const unsigned* nsteps;  // steps finished in this call (nullptr: plain warm start)
  int guess_order;         // 2 quadratic, 1 linear, 0 the last solution
  // inside the device-side WHILE loop, which ends on convergence by itself:
  // the kernels before k_pc_t skip the converged-flag load (the flag can only
  // be raised earlier in the same iteration by a breakdown in k_pc_v, and
  // k_pc_t and k_pc_x, which alone update the solution, still check it)
  bool in_loop;
  const double* minv;
  KS* ks;
  double* partial;
  unsigned* counters;
};

__device__ __forceinline__ bool node_of(const StepArgs& a, int& g, int64_t& pos, int64_t& stride) {
  if (blockIdx.x < a.bm) {
    g = 0;
    pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    stride = a.bm * blockDim.x;
  } else {
    g = 1;
    pos = (blockIdx.x - a.bm) * (int64_t)blockDim.x + threadIdx.x;
    stride = (gridDim.x - a.bm) * (int64_t)blockDim.x;
  }
  return true;
}

__device__ __forceinline__ const double* wslot(const StepArgs& a, int g, int slot) {
  return a.w[g] + (int64_t)slot * a.width[g] * a.count[g];
}
// Weights of an explicit operator application in the type TW it runs in:
// FP64, or FP32 with FP32 sums (the fields and the state stay FP64; each sum
// is rounded to FP64 before it enters the time update).
template <typename TW>
__device__ __forceinline__ const TW* wslot_t(const StepArgs& a, int g, int slot);
template <>
__device__ __forceinline__ const double* wslot_t<double>(const StepArgs& a, int g, int slot) {
  return wslot(a, g, slot);
}
template <>
__device__ __forceinline__ const float* wslot_t<float>(const StepArgs& a, int g, int slot) {
  return a.w32[g] + (int64_t)slot * a.width[g] * a.count[g];
}

// Block-reduce up to 4 partial sums; the last block to finish sums all
// partials in block order and returns true (its thread 0 holds the totals).
template <int Q>
__device__ bool block_done(const StepArgs& a, int which, double (&vals)[Q], double (&tot)[Q]) {
  __shared__ double sh[32][Q];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    double x = vals[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[wid][q] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) / 32;
    for (int q = 0; q < Q; ++q) {
      double x = 0.0;
      for (int i = 0; i < nw; ++i) x += sh[i][q];
      a.partial[((int64_t)which * gridDim.x + blockIdx.x) * 4 + q] = x;
    }
    __threadfence();
    unsigned t = atomicInc(&a.counters[which], gridDim.x - 1);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  // the last block sums every block's partials: thread t takes blocks
  // t, t + blockDim, ... (a fixed order), then the block reduces
  __threadfence();
  double acc[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) acc[q] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] += __ldcg(&a.partial[((int64_t)which * gridDim.x + b) * 4 + q]);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    double x = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[wid][q] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) / 32;
    for (int q = 0; q < Q; ++q) {
      double x = 0.0;
      for (int i = 0; i < nw; ++i) x += sh[i][q];
      tot[q] = x;
    }
  }
  return threadIdx.x == 0;
}

// ---- 1. predictor -----------------------------------------------------------
template <int DIM, typename TW>
__global__ void k_predictor(StepArgs a) {
  int g;
  int64_t pos, stride;
  node_of(a, g, pos, stride);
  const int W = a.width[g];
  const int64_t G = a.count[g];
  for (; pos < G; pos += stride) {
    const int32_t i = a.nodes[g][pos];
    if (a.bc[i] != 0) {
#pragma unroll
      for (int k = 0; k < DIM; ++k) a.vstar[k * a.N + i] = 0.0;
      continue;
    }
    TW grad[DIM][DIM];  // grad[k][j] = d v_k / d x_j
    TW lap[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      lap[k] = TW(0);
#pragma unroll
      for (int j = 0; j < DIM; ++j) grad[k][j] = TW(0);
    }
    const TW* wl = wslot_t<TW>(a, g, a.slot_lap);
    for (int e = 0; e < W; ++e) {
      const int32_t id = a.idx[g][(int64_t)e * G + pos];
      const TW wle = wl[(int64_t)e * G + pos];
      TW wd[DIM];
#pragma unroll
      for (int j = 0; j < DIM; ++j) wd[j] = wslot_t<TW>(a, g, a.slot_d[j])[(int64_t)e * G + pos];
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const TW vk = (TW)a.v[k * a.N + id];
        lap[k] = fma(wle, vk, lap[k]);
#pragma unroll
        for (int j = 0; j < DIM; ++j) grad[k][j] = fma(wd[j], vk, grad[k][j]);
      }
    }
    const double Ti = a.T[i];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      double adv = 0.0;
#pragma unroll
      for (int j = 0; j < DIM; ++j) adv += a.v[j * a.N + i] * (double)grad[k][j];
      double f = -adv + a.Pr * (double)lap[k];
      if (k == DIM - 1) f += a.Ra * a.Pr * (Ti - a.T_ref);
      a.vstar[k * a.N + i] = a.v[k * a.N + i] + a.dt * f;
    }
  }
}

// ---- 2. initial guess of the pressure solve ----------------------------------
// The pressure varies smoothly in time, so the solution of the last three
// steps extrapolated to the new step (quadratic; linear with two) starts the
// solve far closer than the last step's alone: on the seeded 2D sets the
// relative initial residual falls from ~1e-3 to ~1e-7, about half the
// iterations at a 1e-10 tolerance.  The guess only moves the start of the
// iteration; the solve still runs to its tolerance.  Entry N is the border
// unknown c (KS::xN).  Only solutions of the current hsm_step call count as
// history (the incoming p of a call need not be one, e.g. zero from rest):
// at step k of a call, p holds the solution of step k-1 and the history those
// of steps k-2 and k-3, so the guess is linear from k = 2 and quadratic from
// k = 3.
__global__ void k_extrapolate(StepArgs a) {
  const int64_t N1 = a.N + 1;
  const unsigned k = a.nsteps ? *a.nsteps : 0u;
  const int order = a.guess_order;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N1; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = i < a.N ? a.p[i] : a.ks->xN;
    const double h1 = a.hist[i], h2 = a.hist[N1 + i];
    const double g = (order >= 2 && k >= 3u) ? fma(3.0, x - h1, h2) : (order >= 1 && k >= 2u ? fma(2.0, x, -h1) : x);
    a.hist[N1 + i] = h1;
    a.hist[i] = x;
    if (i < a.N)
      a.p[i] = g;
    else
      a.ks->xN = g;
  }
}

// ---- 2a. rhs = div v*/dt, r = rhs - A x0, rhat = r, p = v = 0 ----------------
template <int DIM, typename TW>
__global__ void k_krylov_init(StepArgs a) {
  int g;
  int64_t pos, stride;
  node_of(a, g, pos, stride);
  const int W = a.width[g];
  const int64_t G = a.count[g];
  const int64_t N1 = a.N + 1;
  double* r = a.vec + V_R * N1;
  double* rh = a.vec + V_RHAT * N1;
  double* rhs = a.vec + V_RHS * N1;
  const double xN = a.ks->xN;
  double part[4] = {0.0, 0.0, 0.0, 0.0};  // sum x, sum rhs^2, sum r^2 (rho = rhat.r), 0
  for (; pos < G; pos += stride) {
    const int32_t i = a.nodes[g][pos];
    const bool inner = a.bc[i] == 0;
    TW div = TW(0);
    double ax = 0.0;
    const double* wpg = a.wp[g];
    for (int e = 0; e < W; ++e) {
      const int32_t id = a.idx[g][(int64_t)e * G + pos];
      if (inner) {
#pragma unroll
        for (int k = 0; k < DIM; ++k)
          div = fma(wslot_t<TW>(a, g, a.slot_d[k])[(int64_t)e * G + pos], (TW)a.vstar[k * a.N + id], div);
      }
      ax = fma(wpg[(int64_t)e * G + pos], a.p[id], ax);
    }
    const double b = inner ? (double)div / a.dt : 0.0;
    const double ri = b - (ax + xN);
    rhs[i] = b;
    r[i] = ri;
    rh[i] = ri;
    a.vec[V_P0 * N1 + i] = 0.0;
    a.vec[V_V0 * N1 + i] = 0.0;
    part[0] += a.p[i];
    part[1] += b * b;
    part[2] += ri * ri;
  }
  double tot[4];
  if (block_done<4>(a, 0, part, tot)) {
    KS* ks = a.ks;
    const double rN = 0.0 - tot[0];  // bordered row: 0 - sum x
    r[a.N] = rN;
    rh[a.N] = rN;
    rhs[a.N] = 0.0;
    a.vec[V_P0 * N1 + a.N] = 0.0;
    a.vec[V_V0 * N1 + a.N] = 0.0;
    ks->bnorm2 = tot[1];
    ks->rnorm2 = tot[2] + rN * rN;
    ks->rho = ks->rnorm2;  // rhat = r
    ks->alpha = 1.0;
    ks->omega = 1.0;
    ks->beta = 0.0;
    ks->cur = 0.0;
    ks->iter = 0.0;
    ks->half = 0.0;
    ks->breakdown = 0.0;
    ks->done = (ks->rnorm2 <= ks->tol2 * ks->bnorm2 || ks->bnorm2 == 0.0) ? 1.0 : 0.0;
  }
}

// ---- 2b. one BiCGSTAB iteration in three kernels ---------------------------
// A: p_new = r + beta (p_old - omega v_old) (on the fly), v_new = A p_new,
//    partials: sum p_new, rhat.v_new
template <int DIM>
__global__ void k_bicg_a(StepArgs a) {
  const KS* ks = a.ks;
  if (ks->done != 0.0) return;
  // rho_new = rhat.r is computed by kernel C of the previous iteration; on the
  // first iteration rho_new is the initial r.r (rhat = r)
  int g;
  int64_t pos, stride;
  node_of(a, g, pos, stride);
  const int W = a.width[g];
  const int64_t G = a.count[g];
  const int64_t N1 = a.N + 1;
  const int cur = (int)ks->cur;
  const double* r = a.vec + V_R * N1;
  const double* rh = a.vec + V_RHAT * N1;
  const double* po = a.vec + (cur ? V_P1 : V_P0) * N1;
  const double* vo = a.vec + (cur ? V_V1 : V_V0) * N1;
  double* pn = a.vec + (cur ? V_P0 : V_P1) * N1;
  double* vn = a.vec + (cur ? V_V0 : V_V1) * N1;
  const double beta = ks->beta, omega = ks->omega;
  const double pnN = r[a.N] + beta * (po[a.N] - omega * vo[a.N]);
  double part[2] = {0.0, 0.0};
  for (; pos < G; pos += stride) {
    const int32_t i = a.nodes[g][pos];
    double y = 0.0;
    const double* wpg = a.wp[g];
    for (int e = 0; e < W; ++e) {
      const int32_t id = a.idx[g][(int64_t)e * G + pos];
      const double pj = r[id] + beta * (po[id] - omega * vo[id]);
      y = fma(wpg[(int64_t)e * G + pos], pj * a.minv[id], y);
    }
    y += pnN;
    const double pi = r[i] + beta * (po[i] - omega * vo[i]);
    pn[i] = pi;
    vn[i] = y;
    part[0] += a.minv[i] * pi;
    part[1] += rh[i] * y;
  }
  double tot[2];
  if (block_done<2>(a, 0, part, tot)) {
    KS* k = a.ks;
    pn[a.N] = pnN;
    vn[a.N] = tot[0];
    const double rv = tot[1] + rh[a.N] * tot[0];
    if (rv == 0.0 || !isfinite(rv)) {
      k->breakdown = 1.0;
      k->done = 1.0;
      return;
    }
    k->alpha = k->rho / rv;
    k->cur = 1.0 - k->cur;
  }
}

// B: s = r - alpha v (on the fly), t = A s; partials: sum s, t.s, t.t, s.s
template <int DIM>
__global__ void k_bicg_b(StepArgs a) {
  const KS* ks = a.ks;
  if (ks->done != 0.0) return;
  int g;
  int64_t pos, stride;
  node_of(a, g, pos, stride);
  const int W = a.width[g];
  const int64_t G = a.count[g];
  const int64_t N1 = a.N + 1;
  const int cur = (int)ks->cur;
  const double* r = a.vec + V_R * N1;
  const double* v = a.vec + (cur ? V_V1 : V_V0) * N1;
  double* s = a.vec + V_S * N1;
  double* t = a.vec + V_T * N1;
  const double alpha = ks->alpha;
  const double sN = r[a.N] - alpha * v[a.N];
  double part[4] = {0.0, 0.0, 0.0, 0.0};
  for (; pos < G; pos += stride) {
    const int32_t i = a.nodes[g][pos];
    double y = 0.0;
    const double* wpg = a.wp[g];
    for (int e = 0; e < W; ++e) {
      const int32_t id = a.idx[g][(int64_t)e * G + pos];
      y = fma(wpg[(int64_t)e * G + pos], (r[id] - alpha * v[id]) * a.minv[id], y);
    }
    y += sN;
    const double si = r[i] - alpha * v[i];
    s[i] = si;
    t[i] = y;
    part[0] += a.minv[i] * si;
    part[1] += y * si;
    part[2] += y * y;
    part[3] += si * si;
  }
  double tot[4];
  if (block_done<4>(a, 1, part, tot)) {
    KS* k = a.ks;
    s[a.N] = sN;
    const double tN = tot[0];
    t[a.N] = tN;
    const double ts = tot[1] + tN * sN, tt = tot[2] + tN * tN, ss = tot[3] + sN * sN;
    if (ss <= k->tol2 * k->bnorm2) {
      k->half = 1.0;  // s already small: x += alpha p and stop
      k->omega = 0.0;
    } else if (tt == 0.0 || !isfinite(tt)) {
      k->breakdown = 1.0;
      k->done = 1.0;
    } else {
      k->omega = ts / tt;
    }
  }
}

// C: x += alpha p + omega s, r = s - omega t; partials: rhat.r, r.r
template <int DIM>
__global__ void k_bicg_c(StepArgs a) {
  const KS* ks = a.ks;
  if (ks->done != 0.0) return;
  int g;
  int64_t pos, stride;
  node_of(a, g, pos, stride);
  const int64_t G = a.count[g];
  const int64_t N1 = a.N + 1;
  const int cur = (int)ks->cur;
  double* r = a.vec + V_R * N1;
  const double* rh = a.vec + V_RHAT * N1;
  const double* pc = a.vec + (cur ? V_P1 : V_P0) * N1;
  const double* s = a.vec + V_S * N1;
  const double* t = a.vec + V_T * N1;
  const double alpha = ks->alpha, omega = ks->omega;
  double part[2] = {0.0, 0.0};
  for (; pos < G; pos += stride) {
    const int32_t i = a.nodes[g][pos];
    a.p[i] += a.minv[i] * (alpha * pc[i] + omega * s[i]);
    const double ri = s[i] - omega * t[i];
    r[i] = ri;
    part[0] += rh[i] * ri;
    part[1] += ri * ri;
  }
  double tot[2];
  if (block_done<2>(a, 2, part, tot)) {
    KS* k = a.ks;
    k->xN += alpha * pc[a.N] + omega * s[a.N];
    const double rN = s[a.N] - omega * t[a.N];
    r[a.N] = rN;
    const double rho_new = tot[0] + rh[a.N] * rN;
    k->rnorm2 = tot[1] + rN * rN;
    k->iter += 1.0;
    if (k->half != 0.0 || k->rnorm2 <= k->tol2 * k->bnorm2) {
      k->done = 1.0;
    } else if (rho_new == 0.0 || !isfinite(rho_new) || omega == 0.0) {
      k->breakdown = 1.0;
      k->done = 1.0;
    } else if (k->iter >= k->max_it) {
      k->done = 1.0;
    } else {
      k->beta = (rho_new / k->rho) * (alpha / omega);
      k->rho = rho_new;
    }
  }
}

// ---- 2c. BiCGSTAB right-preconditioned by a multigrid cycle -----------------
// The iterate of the bordered system is (p, c): the pressure field and KS::xN.
// p = r + beta (p - omega v) over all N+1 entries.
__global__ void k_pc_p(StepArgs a) {
  const KS* ks = a.ks;
  if (!a.in_loop && ks->done != 0.0) return;
  const int64_t N1 = a.N + 1;
  const double* r = a.vec + V_R * N1;
  const double* v = a.vec + V_V0 * N1;
  double* pv = a.vec + V_P0 * N1;
  const double beta = ks->beta, omega = ks->omega;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N1; i += (int64_t)gridDim.x * blockDim.x)
    pv[i] = r[i] + beta * (pv[i] - omega * v[i]);
}

// v = A p^ (bordered); alpha = rho / rhat.v
template <int DIM>
__global__ void k_pc_v(StepArgs a) {
  const KS* ks = a.ks;
  if (!a.in_loop && ks->done != 0.0) return;
  int g;
  int64_t pos, stride;
  node_of(a, g, pos, stride);
  const int W = a.width[g];
  const int64_t G = a.count[g];
  const int64_t N1 = a.N + 1;
  const double* ph = a.vec + V_PH * N1;
  const double* rh = a.vec + V_RHAT * N1;
  double* v = a.vec + V_V0 * N1;
  const double phN = ph[a.N];
  double part[2] = {0.0, 0.0};
  for (; pos < G; pos += stride) {
    const int32_t i = a.nodes[g][pos];
    const double* wpg = a.wp[g];
    double y = phN;
    for (int e = 0; e < W; ++e) y = fma(wpg[(int64_t)e * G + pos], ph[a.idx[g][(int64_t)e * G + pos]], y);
    v[i] = y;
    part[0] += ph[i];
    part[1] += rh[i] * y;
  }
  double tot[2];
  if (block_done<2>(a, 0, part, tot)) {
    KS* k = a.ks;
    v[a.N] = tot[0];
    const double rv = tot[1] + rh[a.N] * tot[0];
    if (rv == 0.0 || !isfinite(rv)) {
      k->breakdown = 1.0;
      k->done = 1.0;
      return;
    }
    k->alpha = k->rho / rv;
  }
}

// s = r - alpha v; a small s ends the iteration after x += alpha p^
__global__ void k_pc_s(StepArgs a) {
  const KS* ks = a.ks;
  if (!a.in_loop && ks->done != 0.0) return;
  const int64_t N1 = a.N + 1;
  const double* r = a.vec + V_R * N1;
  const double* v = a.vec + V_V0 * N1;
  double* sv = a.vec + V_S * N1;
  const double alpha = ks->alpha;
  double part[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N1; i += (int64_t)gridDim.x * blockDim.x) {
    const double si = r[i] - alpha * v[i];
    sv[i] = si;
    part[0] += si * si;
  }
  double tot[1];
  if (block_done<1>(a, 1, part, tot)) {
    KS* k = a.ks;
    k->half = tot[0] <= k->tol2 * k->bnorm2 ? 1.0 : 0.0;
  }
}

// t = A s^ (bordered); omega = t.s / t.t
template <int DIM>
__global__ void k_pc_t(StepArgs a) {
  const KS* ks = a.ks;
  if (ks->done != 0.0) return;
  if (ks->half != 0.0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ks->omega = 0.0;
    return;
  }
  int g;
  int64_t pos, stride;
  node_of(a, g, pos, stride);
  const int W = a.width[g];
  const int64_t G = a.count[g];
  const int64_t N1 = a.N + 1;
  const double* sh = a.vec + V_SH * N1;
  const double* sv = a.vec + V_S * N1;
  double* t = a.vec + V_T * N1;
  const double shN = sh[a.N];
  double part[3] = {0.0, 0.0, 0.0};
  for (; pos < G; pos += stride) {
    const int32_t i = a.nodes[g][pos];
    const double* wpg = a.wp[g];
    double y = shN;
    for (int e = 0; e < W; ++e) y = fma(wpg[(int64_t)e * G + pos], sh[a.idx[g][(int64_t)e * G + pos]], y);
    t[i] = y;
    part[0] += sh[i];
    part[1] += y * sv[i];
    part[2] += y * y;
  }
  double tot[3];
  if (block_done<3>(a, 1, part, tot)) {
    KS* k = a.ks;
    const double tN = tot[0];
    t[a.N] = tN;
    const double ts = tot[1] + tN * sv[a.N], tt = tot[2] + tN * tN;
    if (tt == 0.0 || !isfinite(tt)) {
      k->breakdown = 1.0;
      k->done = 1.0;
    } else {
      k->omega = ts / tt;
    }
  }
}

// x += alpha p^ + omega s^, r = s - omega t; rho_new = rhat.r, |r|^2
__global__ void k_pc_x(StepArgs a) {
  const KS* ks = a.ks;
  if (ks->done != 0.0) return;
  const int64_t N1 = a.N + 1;
  double* r = a.vec + V_R * N1;
  const double* rh = a.vec + V_RHAT * N1;
  const double* ph = a.vec + V_PH * N1;
  const double* sh = a.vec + V_SH * N1;
  const double* sv = a.vec + V_S * N1;
  const double* t = a.vec + V_T * N1;
  const double alpha = ks->alpha, omega = ks->omega;
  double part[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.N; i += (int64_t)gridDim.x * blockDim.x) {
    a.p[i] += alpha * ph[i] + omega * sh[i];
    const double ri = sv[i] - omega * t[i];
    r[i] = ri;
    part[0] += rh[i] * ri;
    part[1] += ri * ri;
  }
  double tot[2];
  if (block_done<2>(a, 2, part, tot)) {
    KS* k = a.ks;
    k->xN += alpha * ph[a.N] + omega * sh[a.N];
    const double rN = sv[a.N] - omega * t[a.N];
    r[a.N] = rN;
    const double rho_new = tot[0] + rh[a.N] * rN;
    k->rnorm2 = tot[1] + rN * rN;
    k->iter += 1.0;
    if (k->half != 0.0 || k->rnorm2 <= k->tol2 * k->bnorm2) {
      k->done = 1.0;
    } else if (rho_new == 0.0 || !isfinite(rho_new) || omega == 0.0) {
      k->breakdown = 1.0;
      k->done = 1.0;
    } else if (k->iter >= k->max_it) {
      k->done = 1.0;
    } else {
      k->beta = (rho_new / k->rho) * (alpha / omega);
      k->rho = rho_new;
    }
  }
}

// ---- 2d. GMRES(kGmM) right-preconditioned by the multigrid cycle -------------
// The Arnoldi basis v_0, v_1, ... of the bordered operator B M^-1 (Saad and
// Schultz's GMRES, right-preconditioned: x = x0 + Z y with z_i = M^-1 v_i, and
// y minimising |beta e_1 - H y|), with the Hessenberg matrix reduced by Givens
// rotations as it grows, so that |g_{j+1}| is the residual norm after step j.
// One iteration is one cycle and one operator application: the cycle reads
// vin and writes zout (fixed buffers the captured graph can name; the index j
// lives on the device), the kernels around it copy into and out of the basis.
// Orthogonalisation by classical Gram-Schmidt: the j + 1 dot products in one
// kernel (last-block-done reduction in fixed order), the update and |w| in the
// next.  When the residual meets the tolerance, the basis is full or the
// iteration cap is reached, the small triangular system is solved and x
// updated; a full basis short of the tolerance restarts from the new
// residual.  Those kernels return at once in the other iterations.
constexpr int kGmM = 30;  // restart length
enum { GS_J = 0, GS_FIN = 1, GS_RESTART = 2, GS_HINV = 3, GS_BETA = 4, GS_CONV = 5, GS_H = 8 };
constexpr int GS_CS = GS_H + (kGmM + 1) * kGmM;
constexpr int GS_SN = GS_CS + kGmM;
constexpr int GS_G = GS_SN + kGmM;
constexpr int GS_Y = GS_G + kGmM + 1;
constexpr int GS_SIZE = GS_Y + kGmM;

struct GmArgs {
  double* V;     // [kGmM + 1][N + 1] Arnoldi basis
  double* Z;     // [kGmM][N + 1] its preconditioned images
  double* vin;   // [N + 1] the cycle's input: the current basis vector
  double* zout;  // [N + 1] the cycle's output
  double* w;     // [N + 1]
  double* gs;    // [GS_SIZE] scalars, the Hessenberg matrix (column j at GS_H + j (kGmM + 1)), rotations
  double* part;  // [blocks][kGmM + 1] dot-product partials
  unsigned* cnt; // arrival counter of the dot products
};

__device__ __forceinline__ double& gs_h(double* gs, int i, int j) { return gs[GS_H + j * (kGmM + 1) + i]; }

// after the Krylov set-up: v_0 = r / beta, beta = |r|
__global__ void k_gm_begin(StepArgs a, GmArgs g) {
  const KS* ks = a.ks;
  if (ks->done != 0.0) return;
  const int64_t N1 = a.N + 1;
  const double beta = sqrt(ks->rnorm2), inv = 1.0 / beta;
  const double* r = a.vec + V_R * N1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N1; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = r[i] * inv;
    g.V[i] = v;
    g.vin[i] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    g.gs[GS_J] = 0.0;
    g.gs[GS_FIN] = 0.0;
    g.gs[GS_RESTART] = 0.0;
    g.gs[GS_CONV] = 0.0;
    g.gs[GS_BETA] = beta;
    g.gs[GS_G] = beta;
  }
}

// w = B z (bordered: w_i = (A z)_i + z_N, w_N = sum_i z_i); z_j = z
template <int DIM>
__global__ void k_gm_matvec(StepArgs a, GmArgs g) {
  const KS* ks = a.ks;
  if (!a.in_loop && ks->done != 0.0) return;
  int grp;
  int64_t pos, stride;
  node_of(a, grp, pos, stride);
  const int W = a.width[grp];
  const int64_t G = a.count[grp];
  const int64_t N1 = a.N + 1;
  const int j = (int)g.gs[GS_J];
  const double* z = g.zout;
  double* zj = g.Z + (int64_t)j * N1;
  const double zN = z[a.N];
  double part[1] = {0.0};
  for (; pos < G; pos += stride) {
    const int32_t i = a.nodes[grp][pos];
    const double* wpg = a.wp[grp];
    double y = zN;
    for (int e = 0; e < W; ++e) y = fma(wpg[(int64_t)e * G + pos], z[a.idx[grp][(int64_t)e * G + pos]], y);
    g.w[i] = y;
    const double zi = z[i];
    zj[i] = zi;
    part[0] += zi;
  }
  double tot[1];
  if (block_done<1>(a, 0, part, tot)) {
    g.w[a.N] = tot[0];
    zj[a.N] = zN;
    g.gs[GS_RESTART] = 0.0;  // a restart's basis vector is in place
  }
}

// h_i = v_i . w for i <= j: eight basis vectors per pass over w
__global__ void __launch_bounds__(256) k_gm_dots(StepArgs a, GmArgs g) {
  const KS* ks = a.ks;
  if (!a.in_loop && ks->done != 0.0) return;
  __shared__ double sh[8][8];
  __shared__ bool last;
  const int64_t N1 = a.N + 1;
  const int j = (int)g.gs[GS_J];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i0 = 0; i0 <= j; i0 += 8) {
    double acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N1; k += (int64_t)gridDim.x * blockDim.x) {
      const double wk = g.w[k];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (i0 + u <= j) acc[u] = fma(g.V[(int64_t)(i0 + u) * N1 + k], wk, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      double x = acc[u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) sh[wid][u] = x;
    }
    __syncthreads();
    if (threadIdx.x < 8 && i0 + (int)threadIdx.x <= j) {
      double x = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) x += sh[q][threadIdx.x];
      g.part[(int64_t)blockIdx.x * (kGmM + 1) + i0 + threadIdx.x] = x;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicInc(g.cnt, gridDim.x - 1);
    last = t == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last block sums the partials, eight columns at a time: thread t takes
  // blocks t, t + blockDim, ... (a fixed order), then the block reduces
  for (int i0 = 0; i0 <= j; i0 += 8) {
    double acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (i0 + u <= j) acc[u] += __ldcg(&g.part[(int64_t)b * (kGmM + 1) + i0 + u]);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      double x = acc[u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) sh[wid][u] = x;
    }
    __syncthreads();
    if (threadIdx.x < 8 && i0 + (int)threadIdx.x <= j) {
      double x = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) x += sh[q][threadIdx.x];
      gs_h(g.gs, i0 + threadIdx.x, j) = x;
    }
    __syncthreads();
  }
}

// w -= sum_{i <= j} h_i v_i; |w|; then (last block) the rotations, the
// residual estimate and the decision: continue, or finish this cycle
__global__ void k_gm_update(StepArgs a, GmArgs g) {
  KS* ks = a.ks;
  if (!a.in_loop && ks->done != 0.0) return;
  const int64_t N1 = a.N + 1;
  const int j = (int)g.gs[GS_J];
  double part[1] = {0.0};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N1; k += (int64_t)gridDim.x * blockDim.x) {
    double x = g.w[k];
    for (int i = 0; i <= j; ++i) x = fma(-gs_h(g.gs, i, j), g.V[(int64_t)i * N1 + k], x);
    g.w[k] = x;
    part[0] += x * x;
  }
  double tot[1];
  if (block_done<1>(a, 1, part, tot)) {
    double* gs = g.gs;
    const double hn = sqrt(tot[0]);
    for (int i = 0; i < j; ++i) {
      const double c = gs[GS_CS + i], sn = gs[GS_SN + i];
      const double t0 = c * gs_h(gs, i, j) + sn * gs_h(gs, i + 1, j);
      gs_h(gs, i + 1, j) = -sn * gs_h(gs, i, j) + c * gs_h(gs, i + 1, j);
      gs_h(gs, i, j) = t0;
    }
    const double hjj = gs_h(gs, j, j);
    const double den = hypot(hjj, hn);
    if (den == 0.0 || !isfinite(den)) {
      ks->breakdown = 1.0;
      ks->done = 1.0;
      gs[GS_FIN] = 0.0;
      return;
    }
    const double c = hjj / den, sn = hn / den;
    gs[GS_CS + j] = c;
    gs[GS_SN + j] = sn;
    gs_h(gs, j, j) = den;
    const double gj = gs[GS_G + j];
    gs[GS_G + j + 1] = -sn * gj;
    gs[GS_G + j] = c * gj;
    ks->iter += 1.0;
    const double res2 = gs[GS_G + j + 1] * gs[GS_G + j + 1];
    ks->rnorm2 = res2;
    const bool conv = res2 <= ks->tol2 * ks->bnorm2 || hn == 0.0;
    const bool fin = conv || j + 1 == kGmM || ks->iter >= ks->max_it;
    gs[GS_CONV] = conv ? 1.0 : 0.0;
    gs[GS_FIN] = fin ? 1.0 : 0.0;
    if (!fin) {
      gs[GS_J] = (double)(j + 1);
      gs[GS_HINV] = 1.0 / hn;
    }
  }
}

// v_{j+1} = w / h_{j+1,j}, also the next cycle's input
__global__ void k_gm_next(StepArgs a, GmArgs g) {
  const KS* ks = a.ks;
  if (ks->done != 0.0 || g.gs[GS_FIN] != 0.0) return;
  const int64_t N1 = a.N + 1;
  const int j = (int)g.gs[GS_J];
  const double hinv = g.gs[GS_HINV];
  double* vj = g.V + (int64_t)j * N1;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N1; k += (int64_t)gridDim.x * blockDim.x) {
    const double v = g.w[k] * hinv;
    vj[k] = v;
    g.vin[k] = v;
  }
}

// end of a cycle: y = R^-1 g (R the rotated Hessenberg matrix, upper triangular)
__global__ void k_gm_solve(StepArgs a, GmArgs g) {
  if (a.ks->done != 0.0 || g.gs[GS_FIN] == 0.0 || threadIdx.x != 0) return;
  double* gs = g.gs;
  const int jj = (int)gs[GS_J] + 1;
  for (int i = jj - 1; i >= 0; --i) {
    double s = gs[GS_G + i];
    for (int k = i + 1; k < jj; ++k) s = fma(-gs_h(gs, i, k), gs[GS_Y + k], s);
    gs[GS_Y + i] = s / gs_h(gs, i, i);
  }
}

// x += Z y; then the solve is done, or restarts from the new residual
__global__ void k_gm_x(StepArgs a, GmArgs g) {
  KS* ks = a.ks;
  if (ks->done != 0.0 || g.gs[GS_FIN] == 0.0) return;
  const int64_t N1 = a.N + 1;
  const double* gs = g.gs;
  const int jj = (int)gs[GS_J] + 1;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N1; k += (int64_t)gridDim.x * blockDim.x) {
    double x = 0.0;
    for (int t = 0; t < jj; ++t) x = fma(gs[GS_Y + t], g.Z[(int64_t)t * N1 + k], x);
    if (k < a.N)
      a.p[k] += x;
    else
      ks->xN += x;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (gs[GS_CONV] != 0.0 || ks->iter >= ks->max_it)
      ks->done = 1.0;
    else
      g.gs[GS_RESTART] = 1.0;
  }
}

// restart: r = rhs - B x into v_0 (unscaled), beta = |r|
template <int DIM>
__global__ void k_gm_restart(StepArgs a, GmArgs g) {
  KS* ks = a.ks;
  if (ks->done != 0.0 || g.gs[GS_RESTART] == 0.0) return;
  int grp;
  int64_t pos, stride;
  node_of(a, grp, pos, stride);
  const int W = a.width[grp];
  const int64_t G = a.count[grp];
  const int64_t N1 = a.N + 1;
  const double* rhs = a.vec + V_RHS * N1;
  const double xN = ks->xN;
  double part[2] = {0.0, 0.0};
  for (; pos < G; pos += stride) {
    const int32_t i = a.nodes[grp][pos];
    const double* wpg = a.wp[grp];
    double y = xN;
    for (int e = 0; e < W; ++e) y = fma(wpg[(int64_t)e * G + pos], a.p[a.idx[grp][(int64_t)e * G + pos]], y);
    const double ri = rhs[i] - y;
    g.V[i] = ri;
    part[0] += a.p[i];
    part[1] += ri * ri;
  }
  double tot[2];
  if (block_done<2>(a, 2, part, tot)) {
    double* gs = g.gs;
    const double rN = 0.0 - tot[0];
    g.V[a.N] = rN;
    const double beta = sqrt(tot[1] + rN * rN);
    gs[GS_BETA] = beta;
    gs[GS_G] = beta;
    gs[GS_J] = 0.0;
    gs[GS_FIN] = 0.0;
    gs[GS_CONV] = 0.0;
  }
}

// restart: v_0 /= beta, also the next cycle's input
__global__ void k_gm_rscale(StepArgs a, GmArgs g) {
  const KS* ks = a.ks;
  if (ks->done != 0.0 || g.gs[GS_RESTART] == 0.0) return;
  const int64_t N1 = a.N + 1;
  const double inv = 1.0 / g.gs[GS_BETA];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N1; k += (int64_t)gridDim.x * blockDim.x) {
    const double v = g.V[k] * inv;
    g.V[k] = v;
    g.vin[k] = v;
  }
}

// ---- 3. correction and 4. temperature ----------------------------------------
template <int DIM, typename TW>
__global__ void k_correct_temperature(StepArgs a) {
  int g;
  int64_t pos, stride;
  node_of(a, g, pos, stride);
  const int W = a.width[g];
  const int64_t G = a.count[g];
  for (; pos < G; pos += stride) {
    const int32_t i = a.nodes[g][pos];
    const uint8_t b = a.bc[i];
    if (b != 0) {
#pragma unroll
      for (int k = 0; k < DIM; ++k) a.v[k * a.N + i] = 0.0;
      a.Tn[i] = b == HSM_BC_T_DIRICHLET ? a.T_bc[i] : a.T[i];
      continue;
    }
    TW gp[DIM], gT[DIM], lT = TW(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) gp[k] = gT[k] = TW(0);
    const TW* wl = wslot_t<TW>(a, g, a.slot_lap);
    for (int e = 0; e < W; ++e) {
      const int32_t id = a.idx[g][(int64_t)e * G + pos];
      const TW pj = (TW)a.p[id], Tj = (TW)a.T[id];
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const TW wd = wslot_t<TW>(a, g, a.slot_d[k])[(int64_t)e * G + pos];
        gp[k] = fma(wd, pj, gp[k]);
        gT[k] = fma(wd, Tj, gT[k]);
      }
      lT = fma(wl[(int64_t)e * G + pos], Tj, lT);
    }
    double adv = 0.0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const double vk = a.vstar[k * a.N + i] - a.dt * (double)gp[k];
      a.v[k * a.N + i] = vk;
      adv += vk * (double)gT[k];
    }
    a.Tn[i] = a.T[i] + a.dt * (-adv + (double)lT);
  }
}

// ---- 5. temperature boundary closure and write-back -------------------------
__global__ void k_temperature_bc(StepArgs a) {
  int g;
  int64_t pos, stride;
  node_of(a, g, pos, stride);
  const int W = a.width[g];
  const int64_t G = a.count[g];
  for (; pos < G; pos += stride) {
    const int32_t i = a.nodes[g][pos];
    double Ti = a.Tn[i];
    if (g == 1 && a.bc[i] == HSM_BC_T_NEUMANN) {
      const double* wn = a.wn[1];
      double s = 0.0;
      for (int e = 1; e < W; ++e) s = fma(wn[(int64_t)e * G + pos], a.Tn[a.idx[1][(int64_t)e * G + pos]], s);
      Ti = -s / wn[pos];
    }
    a.T[i] = Ti;
  }
}

// Pressure-row and wall normal-derivative weights of the RBF-FD group.
template <int DIM>
__global__ void k_wall_weights(const int32_t* __restrict__ nodes, int64_t G, int W, const double* __restrict__ w,
                               int s0, int s1, int s2, int slap, const uint8_t* __restrict__ bc,
                               const double* __restrict__ normals, int64_t N, double* wp, double* wn) {
  const int slots[3] = {s0, s1, s2};
  for (int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pos < G; pos += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = nodes[pos];
    const bool wall = bc[i] != 0;
    for (int e = 0; e < W; ++e) {
      double x = 0.0;
#pragma unroll
      for (int k = 0; k < DIM; ++k) x = fma(normals[k * N + i], w[((int64_t)slots[k] * W + e) * G + pos], x);
      wn[(int64_t)e * G + pos] = wall ? x : 0.0;
      wp[(int64_t)e * G + pos] = wall ? x : w[((int64_t)slap * W + e) * G + pos];
    }
  }
}

// Jacobi preconditioner: inverse of the centre weight of every pressure row
// (the centre is the first stencil entry of both groups).
__global__ void k_minv(StepArgs a) {
  int g;
  int64_t pos, stride;
  node_of(a, g, pos, stride);
  const int64_t G = a.count[g];
  double* minv = const_cast<double*>(a.minv);
  for (; pos < G; pos += stride) {
    const double d = a.wp[g][pos];
    minv[a.nodes[g][pos]] = (d != 0.0 && isfinite(d)) ? 1.0 / d : 1.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) minv[a.N] = 1.0;
}

StepArgs make_args(hsm_stepper st, double* v, double* T, double* p) {
  hsm_plan pl = st->plan;
  StepArgs a{};
  a.nodes[0] = pl->mon.nodes;
  a.nodes[1] = pl->rbf.nodes;
  a.idx[0] = pl->mon.idx;
  a.idx[1] = pl->rbf.idx;
  a.w[0] = pl->mon.w64;
  a.w[1] = pl->rbf.w64;
  a.w32[0] = pl->mon.w32;
  a.w32[1] = pl->rbf.w32;
  a.wp[0] = pl->mon.w64 + (int64_t)st->slot_lap * pl->mon.width * pl->mon.count;
  a.wp[1] = st->wp_rbf;
  a.wn[0] = nullptr;
  a.wn[1] = st->wn_rbf;
  a.count[0] = pl->mon.count;
  a.count[1] = pl->rbf.count;
  a.width[0] = pl->mon.width;
  a.width[1] = pl->rbf.width;
  a.bm = st->blocks_mon;
  for (int k = 0; k < 3; ++k) a.slot_d[k] = st->slot_d[k];
  a.slot_lap = st->slot_lap;
  a.dim = st->dim;
  a.N = st->N;
  a.Ra = st->phys.Ra;
  a.Pr = st->phys.Pr;
  a.dt = st->phys.dt;
  a.T_ref = st->phys.T_ref;
  a.bc = st->phys.bc;
  a.T_bc = st->phys.T_bc;
  a.v = v;
  a.T = T;
  a.p = p;
  a.vstar = st->vstar;
  a.Tn = st->Tn;
  a.vec = st->vec;
  a.hist = st->hist;
  a.nsteps = nullptr;
  a.guess_order = st->phys.guess_order == 0 ? 2 : (st->phys.guess_order == 1 ? 1 : 0);
  a.minv = st->minv;
  a.ks = reinterpret_cast<KS*>(st->scal);
  a.partial = st->partial;
  a.counters = st->counters;
  return a;
}

// Device side of the conditional Krylov loop.  Every pass of the loop body
// ends with k_loop_cond, which keeps the loop going while the solve has not
// converged; a pass counter caps the loop at cap passes, so it always ends.
// Before the loop: reset the pass counter and open the loop only if the
// set-up has not already met the tolerance (a good initial guess can), so
// the body never runs on a converged solve.
__global__ void k_loop_begin(const KS* ks, unsigned* ctl, cudaGraphConditionalHandle h) {
  ctl[0] = 0u;
  cudaGraphSetConditional(h, ks->done == 0.0 ? 1u : 0u);
}

__global__ void k_loop_cond(const KS* ks, unsigned* ctl, unsigned cap, cudaGraphConditionalHandle h) {
  const unsigned c = ++ctl[0];
  const bool open = ks->done == 0.0;
  if (open && c >= cap) ctl[2] = 1u;
  cudaGraphSetConditional(h, open && c < cap ? 1u : 0u);
}

// Iterations and convergence of the step that just finished.
__global__ void k_step_record(const KS* ks, unsigned* ctl, int* iters, int* bad, int cap) {
  const unsigned k = ctl[1]++;
  if ((int)k < cap) {
    iters[k] = (int)ks->iter;
    bad[k] = (ks->breakdown != 0.0 || ks->rnorm2 > ks->tol2 * ks->bnorm2 * 1.0000001) ? 1 : 0;
  }
}

// The explicit operator applications in FP64 or, with hsm_phys.apply_f32,
// FP32 weights and sums.
template <int DIM>
void launch_predictor(hsm_stepper st, const StepArgs& a, dim3 grid, dim3 blk, cudaStream_t s) {
  if (st->phys.apply_f32)
    k_predictor<DIM, float><<<grid, blk, 0, s>>>(a);
  else
    k_predictor<DIM, double><<<grid, blk, 0, s>>>(a);
}
GmArgs make_gm(hsm_stepper st);
template <int DIM>
void launch_krylov_init(hsm_stepper st, const StepArgs& a, dim3 grid, dim3 blk, cudaStream_t s) {
  if (st->phys.apply_f32)
    k_krylov_init<DIM, float><<<grid, blk, 0, s>>>(a);
  else
    k_krylov_init<DIM, double><<<grid, blk, 0, s>>>(a);
  if (st->gmres) k_gm_begin<<<grid, blk, 0, s>>>(a, make_gm(st));
}
template <int DIM>
void launch_correct_temperature(hsm_stepper st, const StepArgs& a, dim3 grid, dim3 blk, cudaStream_t s) {
  if (st->phys.apply_f32)
    k_correct_temperature<DIM, float><<<grid, blk, 0, s>>>(a);
  else
    k_correct_temperature<DIM, double><<<grid, blk, 0, s>>>(a);
}

// Krylov iterations per captured chunk: Jacobi needs thousands of iterations
// per solve, the multigrid preconditioner tens, each of ~50 kernels.
int chunk_iters(hsm_stepper st) { return st->amg ? 2 : 16; }
int chunk_kernels(hsm_stepper st) {
  if (st->gmres) return chunk_iters(st) * (8 + amg_kernels_per_cycle(*st->amg));
  return st->amg ? chunk_iters(st) * (5 + 2 * amg_kernels_per_cycle(*st->amg)) : chunk_iters(st) * 3;
}

GmArgs make_gm(hsm_stepper st) {
  const int64_t N1 = st->N + 1;
  GmArgs g{};
  g.V = st->gm_vec;
  g.Z = g.V + (int64_t)(kGmM + 1) * N1;
  g.vin = g.Z + (int64_t)kGmM * N1;
  g.zout = g.vin + N1;
  g.w = g.zout + N1;
  g.gs = st->gm_scal;
  g.part = st->gm_part;
  g.cnt = st->gm_cnt;
  return g;
}

template <int DIM>
void launch_iters(hsm_stepper st, const StepArgs& a, dim3 grid, dim3 blk, cudaStream_t s, int n_iters) {
  const int64_t N1 = a.N + 1;
  for (int c = 0; c < n_iters; ++c) {
    if (st->gmres) {
      const double* done = a.in_loop ? nullptr : &a.ks->done;
      const GmArgs g = make_gm(st);
      amg_vcycle(*st->amg, g.vin, g.zout, done, s);
      k_gm_matvec<DIM><<<grid, blk, 0, s>>>(a, g);
      k_gm_dots<<<grid, blk, 0, s>>>(a, g);
      k_gm_update<<<grid, blk, 0, s>>>(a, g);
      k_gm_next<<<grid, blk, 0, s>>>(a, g);
      k_gm_solve<<<1, 32, 0, s>>>(a, g);
      k_gm_x<<<grid, blk, 0, s>>>(a, g);
      k_gm_restart<DIM><<<grid, blk, 0, s>>>(a, g);
      k_gm_rscale<<<grid, blk, 0, s>>>(a, g);
    } else if (st->amg) {
      const double* done = a.in_loop ? nullptr : &a.ks->done;
      k_pc_p<<<grid, blk, 0, s>>>(a);
      amg_vcycle(*st->amg, a.vec + V_P0 * N1, a.vec + V_PH * N1, done, s);
      k_pc_v<DIM><<<grid, blk, 0, s>>>(a);
      k_pc_s<<<grid, blk, 0, s>>>(a);
      amg_vcycle(*st->amg, a.vec + V_S * N1, a.vec + V_SH * N1, done, s);
      k_pc_t<DIM><<<grid, blk, 0, s>>>(a);
      k_pc_x<<<grid, blk, 0, s>>>(a);
    } else {
      k_bicg_a<DIM><<<grid, blk, 0, s>>>(a);
      k_bicg_b<DIM><<<grid, blk, 0, s>>>(a);
      k_bicg_c<DIM><<<grid, blk, 0, s>>>(a);
    }
  }
}

template <int DIM>
void launch_chunk(hsm_stepper st, const StepArgs& a, dim3 grid, dim3 blk, cudaStream_t s) {
  launch_iters<DIM>(st, a, grid, blk, s, chunk_iters(st));
}

template <typename F>
cudaError_t capture(cudaStream_t s, cudaGraphExec_t* out, F&& body) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  body();
  e = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e;
}

void drop_graphs(hsm_stepper st) {
  for (cudaGraphExec_t* g : {&st->g_head, &st->g_chunk, &st->g_tail, &st->g_step})
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
  st->head_chunks = 0;
}

// One step as one graph: predictor, Krylov set-up, the Krylov iterations in
// a conditional WHILE node (body: one iteration and k_loop_cond), correction,
// temperature and the record of the step's iteration count.
template <int DIM>
cudaError_t capture_step(hsm_stepper st, const StepArgs& a, dim3 grid, dim3 blk, cudaStream_t cs, cudaStream_t bs,
                         cudaGraphExec_t* out) {
  const unsigned cap = (unsigned)st->phys.krylov_max_it + 2u;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  launch_predictor<DIM>(st, a, grid, blk, cs);
  {
    StepArgs ax = a;
    ax.nsteps = st->ctl + 1;  // k_step_record counts the steps of the call
    k_extrapolate<<<grid, blk, 0, cs>>>(ax);
  }
  launch_krylov_init<DIM>(st, a, grid, blk, cs);
  cudaStreamCaptureStatus status;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaGraphConditionalHandle h{};
  cudaGraphNode_t cnode = nullptr;
  cudaGraphNodeParams np = {};
  e = cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, &deps, nullptr, &ndeps);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, cg, 0u, 0u);
  if (e == cudaSuccess) {
    k_loop_begin<<<1, 1, 0, cs>>>(a.ks, st->ctl, h);
    e = cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, &deps, nullptr, &ndeps);
  }
  if (e == cudaSuccess) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&cnode, cg, deps, nullptr, ndeps, &np);
  }
  if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e == cudaSuccess) {
    // the loop body, captured on a second stream into the node's graph
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      StepArgs al = a;
      al.in_loop = true;
      launch_iters<DIM>(st, al, grid, blk, bs, 1);
      k_loop_cond<<<1, 1, 0, bs>>>(a.ks, st->ctl, cap, h);
      e = cudaStreamEndCapture(bs, &body);
    }
  }
  if (e == cudaSuccess) {
    launch_correct_temperature<DIM>(st, a, grid, blk, cs);
    k_temperature_bc<<<grid, blk, 0, cs>>>(a);
    k_step_record<<<1, 1, 0, cs>>>(a.ks, st->ctl, st->step_iters, st->step_bad, st->step_cap);
  }
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  return e;
}

// Each step runs as CUDA graphs: the head graph (predictor, Krylov set-up and
// enough Krylov chunks for the previous step's iteration count plus one
// chunk) is launched, the solver state is read once, further chunk graphs run
// only if the solve has not converged, then the tail graph finishes the step.
// Chunks after convergence cost only their launches: every Krylov kernel
// returns at once when the converged flag is set.
template <int DIM>
hsm_status run_steps(hsm_stepper st, int n_steps, double* v, double* T, double* p, int* iters, bool* notconv) {
  hsm_plan pl = st->plan;
  cudaStream_t s = pl->stream;
  StepArgs a = make_args(st, v, T, p);
  const dim3 grid((unsigned)(st->blocks_mon + st->blocks_rbf)), blk(st->threads);
  if (st->gv != v || st->gT != T || st->gp != p) {
    drop_graphs(st);
    st->gv = v;
    st->gT = T;
    st->gp = p;
  }
  // graphs are captured on a private stream (capture is not possible on the
  // legacy default stream) and launched on the plan's stream
  if (!st->cap) HSM_CUDA(pl, cudaStreamCreateWithFlags(&st->cap, cudaStreamNonBlocking));
  cudaStream_t cs = st->cap;
  // The caller owns p, the stepper only the bordering constant c: a c left by
  // an earlier call need not match the p passed now (a reset or restarted
  // run), and with a near-zero right-hand side (a first step from rest) the
  // solve could not then reach its relative tolerance.  Each call starts c
  // at zero; within a call every solve is warm-started from the last.
  HSM_CUDA(pl, cudaMemsetAsync(reinterpret_cast<char*>(st->scal) + offsetof(KS, xN), 0, sizeof(double), s));
  // the grid barrier of the cooperative multigrid cycle starts each call clear
  const unsigned* tflag = st->amg ? amg_timeout_flag(*st->amg) : nullptr;
  unsigned timed_out = 0;
  if (st->amg) HSM_CUDA(pl, amg_reset_barrier(*st->amg, s));
  if (!st->g_chunk) HSM_CUDA(pl, capture(cs, &st->g_chunk, [&] { launch_chunk<DIM>(st, a, grid, blk, cs); }));
  if (!st->g_tail)
    HSM_CUDA(pl, capture(cs, &st->g_tail, [&] {
      launch_correct_temperature<DIM>(st, a, grid, blk, cs);
      k_temperature_bc<<<grid, blk, 0, cs>>>(a);
    }));
  // device-side loop: one graph launch per step, one synchronisation per call
  if (!st->g_step_failed) {
    if (n_steps > st->step_cap) {
      dev_free(&st->step_iters, s);
      dev_free(&st->step_bad, s);
      drop_graphs(st);
      const int cap = std::max(n_steps, 64);
      HSM_CUDA(pl, dev_alloc(&st->step_iters, cap, s));
      HSM_CUDA(pl, dev_alloc(&st->step_bad, cap, s));
      st->step_cap = cap;
    }
    if (!st->ctl) HSM_CUDA(pl, dev_alloc(&st->ctl, 4, s));
    if (!st->g_step) {
      if (!st->body) HSM_CUDA(pl, cudaStreamCreateWithFlags(&st->body, cudaStreamNonBlocking));
      if (capture_step<DIM>(st, a, grid, blk, cs, st->body, &st->g_step) != cudaSuccess) {
        // conditional graph nodes are not available here: clear the error and
        // fall back to the host-driven loop below
        cudaGetLastError();
        st->g_step = nullptr;
        st->g_step_failed = true;
      }
    }
  }
  if (st->g_step) {
    HSM_CUDA(pl, cudaMemsetAsync(st->ctl, 0, 4 * sizeof(unsigned), s));
    for (int it = 0; it < n_steps; ++it) {
      HSM_CUDA(pl, cudaGraphLaunch(st->g_step, s));
      pl->launches += 7;
    }
    std::vector<int> it_h(n_steps > 0 ? n_steps : 1), bad_h(n_steps > 0 ? n_steps : 1);
    unsigned ctl_h[4] = {0, 0, 0, 0};
    if (n_steps > 0) {
      HSM_CUDA(pl, cudaMemcpyAsync(it_h.data(), st->step_iters, n_steps * sizeof(int), cudaMemcpyDeviceToHost, s));
      HSM_CUDA(pl, cudaMemcpyAsync(bad_h.data(), st->step_bad, n_steps * sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    HSM_CUDA(pl, cudaMemcpyAsync(ctl_h, st->ctl, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    if (tflag) HSM_CUDA(pl, cudaMemcpyAsync(&timed_out, tflag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    HSM_CUDA(pl, cudaStreamSynchronize(s));
    if (timed_out) return set_error(pl, HSM_ETIMEOUT, "a grid barrier of the multigrid cycle timed out");
    for (int it = 0; it < n_steps; ++it) {
      if (iters) iters[it] = it_h[it];
      if (bad_h[it]) *notconv = true;
      pl->launches += (int64_t)it_h[it] * (chunk_kernels(st) / chunk_iters(st) + 1);
    }
    if (ctl_h[2]) *notconv = true;
    if (n_steps > 0) st->last_iters = it_h[n_steps - 1];
    return HSM_OK;
  }
  KS host{};
  const int kChunk = chunk_iters(st);
  const int max_chunks = (int)(st->phys.krylov_max_it / kChunk) + 2;
  for (int it = 0; it < n_steps; ++it) {
    const int want = std::min(max_chunks, (st->last_iters + kChunk - 1) / kChunk + 1);
    if (!st->g_head || st->head_chunks != want) {
      if (st->g_head) cudaGraphExecDestroy(st->g_head);
      st->g_head = nullptr;
      HSM_CUDA(pl, capture(cs, &st->g_head, [&] {
        launch_predictor<DIM>(st, a, grid, blk, cs);
        launch_krylov_init<DIM>(st, a, grid, blk, cs);
        for (int c = 0; c < want; ++c) launch_chunk<DIM>(st, a, grid, blk, cs);
      }));
      st->head_chunks = want;
    }
    HSM_CUDA(pl, cudaGraphLaunch(st->g_head, s));
    pl->launches += 2 + chunk_kernels(st) * want;
    int done_chunks = want;
    for (;;) {
      HSM_CUDA(pl, cudaMemcpyAsync(&host, a.ks, sizeof(KS), cudaMemcpyDeviceToHost, s));
      HSM_CUDA(pl, cudaStreamSynchronize(s));
      if (host.done != 0.0 || done_chunks >= max_chunks) break;
      HSM_CUDA(pl, cudaGraphLaunch(st->g_chunk, s));
      pl->launches += chunk_kernels(st);
      ++done_chunks;
    }
    st->last_iters = (int)host.iter;
    if (iters) iters[it] = (int)host.iter;
    if (host.breakdown != 0.0 || host.rnorm2 > host.tol2 * host.bnorm2 * 1.0000001) *notconv = true;
    HSM_CUDA(pl, cudaGraphLaunch(st->g_tail, s));
    pl->launches += 2;
  }
  if (tflag) HSM_CUDA(pl, cudaMemcpyAsync(&timed_out, tflag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  HSM_CUDA(pl, cudaStreamSynchronize(s));
  if (timed_out) return set_error(pl, HSM_ETIMEOUT, "a grid barrier of the multigrid cycle timed out");
  return HSM_OK;
}

}  // namespace
}  // namespace hsm

using namespace hsm;

extern "C" {

hsm_status hsm_stepper_create(hsm_stepper* out, hsm_plan pl, const hsm_phys* phys) {
  if (!out || !pl || !phys) return set_error(pl, HSM_EINVAL, "out, plan and phys are required");
  *out = nullptr;
  if (!pl->weights_built) return set_error(pl, HSM_ESTATE, "the plan's weights are not computed");
  {
    const hsm_status ck = check_gate(pl);
    if (ck != HSM_OK) return ck;
  }
  const unsigned need = HSM_DX | HSM_DY | HSM_LAP | (pl->dim == 3 ? HSM_DZ : 0);
  if ((pl->op_mask & need) != need) return set_error(pl, HSM_EINVAL, "the plan needs every first derivative and the Laplacian");
  if (!phys->bc || !phys->T_bc || !phys->normals) return set_error(pl, HSM_EINVAL, "bc, T_bc and normals are required");
  if (!(phys->dt > 0.0) || !(phys->krylov_tol > 0.0) || phys->krylov_max_it < 1)
    return set_error(pl, HSM_EINVAL, "dt, krylov_tol and krylov_max_it must be positive");
  if (phys->guess_order < -1 || phys->guess_order > 1)
    return set_error(pl, HSM_EINVAL, "guess_order must be -1, 0 or 1");
  if (phys->apply_f32 != 0 && phys->apply_f32 != 1) return set_error(pl, HSM_EINVAL, "apply_f32 must be 0 or 1");
  if (phys->mg_tail_from < -1 || phys->mg_fused_from < -1)
    return set_error(pl, HSM_EINVAL, "mg_tail_from and mg_fused_from must be >= -1");
  if (phys->mg_persistent < -1 || phys->mg_persistent > 1)
    return set_error(pl, HSM_EINVAL, "mg_persistent must be -1, 0 or 1");
  if (phys->mg_sweeps < 0 || phys->mg_sweeps > 2) return set_error(pl, HSM_EINVAL, "mg_sweeps must be 0, 1 or 2");
  if (phys->krylov != HSM_KRYLOV_BICGSTAB && phys->krylov != HSM_KRYLOV_GMRES)
    return set_error(pl, HSM_EINVAL, "unknown Krylov method");
  if (phys->precond != HSM_PRECOND_AMG && phys->precond != HSM_PRECOND_JACOBI)
    return set_error(pl, HSM_EINVAL, "unknown preconditioner");
  if (phys->apply_f32 && (!pl->mon.w32 || !pl->rbf.w32)) {
    // FP32 copies of the plan's weights, as hsm_apply(HSM_F32) makes them
    HSM_CUDA(pl, dev_alloc(&pl->mon.w32, (size_t)pl->nops * pl->mon.width * pl->mon.count, pl->stream));
    HSM_CUDA(pl, dev_alloc(&pl->rbf.w32, (size_t)pl->nops * pl->rbf.width * pl->rbf.count, pl->stream));
    const hsm_status ws = weights_to_f32(pl);
    if (ws != HSM_OK) return ws;
  }
  hsm_stepper st = new (std::nothrow) hsm_stepper_s();
  if (!st) return set_error(pl, HSM_ENOMEM, "host allocation failed");
  st->plan = pl;
  st->phys = *phys;
  st->dim = pl->dim;
  st->N = pl->N;
  int slot = 0;
  for (int b = 0; b < 4; ++b) {
    if (!(pl->op_mask & (1u << b))) continue;
    if (b < 3) st->slot_d[b] = slot;
    else st->slot_lap = slot;
    ++slot;
  }
  cudaStream_t s = pl->stream;
  auto fail = [&](hsm_status code) {
    hsm_stepper_destroy(st);
    return code;
  };
  const int64_t N = pl->N, G = pl->rbf.count, W = pl->rbf.width;
  if (dev_alloc(&st->wp_rbf, W * G, s) || dev_alloc(&st->wn_rbf, W * G, s) ||
      dev_alloc(&st->vstar, (size_t)pl->dim * N, s) || dev_alloc(&st->Tn, N, s) || dev_alloc(&st->minv, N + 1, s) ||
      dev_alloc(&st->vec, (size_t)V_COUNT * (N + 1), s) || dev_alloc(&st->hist, (size_t)2 * (N + 1), s) ||
      dev_alloc(&st->scal, 16, s))
    return fail(set_error(pl, HSM_ENOMEM, "stepper allocation failed"));
  const int T = st->threads;
  const int64_t full = (int64_t)num_sms() * (2048 / T);
  const int64_t tot = pl->mon.count + pl->rbf.count;
  st->blocks_mon = pl->mon.count ? (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(pl->mon.count, T),
                                                                                 full * pl->mon.count / tot + 1))
                                 : 0;
  st->blocks_rbf = pl->rbf.count ? (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(pl->rbf.count, T),
                                                                                 full * pl->rbf.count / tot + 1))
                                 : 0;
  const int nb = st->blocks_mon + st->blocks_rbf;
  if (dev_alloc(&st->partial, (size_t)3 * nb * 4, s) || dev_alloc(&st->counters, 4, s))
    return fail(set_error(pl, HSM_ENOMEM, "stepper allocation failed"));
  st->gmres = phys->precond == HSM_PRECOND_AMG && phys->krylov == HSM_KRYLOV_GMRES;
  if (st->gmres) {
    if (dev_alloc(&st->gm_vec, (size_t)(2 * kGmM + 4) * (N + 1), s) || dev_alloc(&st->gm_scal, GS_SIZE, s) ||
        dev_alloc(&st->gm_part, (size_t)nb * (kGmM + 1), s) || dev_alloc(&st->gm_cnt, 1, s))
      return fail(set_error(pl, HSM_ENOMEM, "stepper allocation failed"));
    if (cudaMemsetAsync(st->gm_cnt, 0, sizeof(unsigned), s) != cudaSuccess ||
        cudaMemsetAsync(st->gm_scal, 0, GS_SIZE * sizeof(double), s) != cudaSuccess)
      return fail(set_error(pl, HSM_ECUDA, "memset failed"));
  }
  if (cudaMemsetAsync(st->counters, 0, 4 * sizeof(unsigned), s) != cudaSuccess)
    return fail(set_error(pl, HSM_ECUDA, "memset failed"));
  KS ks{};
  ks.tol2 = phys->krylov_tol * phys->krylov_tol;
  ks.max_it = phys->krylov_max_it;
  ks.xN = 0.0;
  ks.done = 1.0;
  if (cudaMemcpyAsync(st->scal, &ks, sizeof(KS), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return fail(set_error(pl, HSM_ECUDA, "copy failed"));
  if (G) {
    int grid = (int)std::min<int64_t>(ceil_div(G, 256), (int64_t)num_sms() * 8);
    if (pl->dim == 2)
      k_wall_weights<2><<<grid, 256, 0, s>>>(pl->rbf.nodes, G, (int)W, pl->rbf.w64, st->slot_d[0], st->slot_d[1], 0,
                                             st->slot_lap, phys->bc, phys->normals, N, st->wp_rbf, st->wn_rbf);
    else
      k_wall_weights<3><<<grid, 256, 0, s>>>(pl->rbf.nodes, G, (int)W, pl->rbf.w64, st->slot_d[0], st->slot_d[1],
                                             st->slot_d[2], st->slot_lap, phys->bc, phys->normals, N, st->wp_rbf,
                                             st->wn_rbf);
  }
  {
    StepArgs a = make_args(st, nullptr, nullptr, nullptr);
    k_minv<<<st->blocks_mon + st->blocks_rbf, st->threads, 0, s>>>(a);
    if (phys->precond == HSM_PRECOND_AMG) {
      st->amg = new (std::nothrow) Amg();
      if (!st->amg) return fail(set_error(pl, HSM_ENOMEM, "host allocation failed"));
      // over-correction of the coarse-grid step (2^d nodes per aggregate)
      hsm_status as = amg_setup(pl, a.wp[0], a.wp[1], pl->dim == 2 ? 1.8 : 1.5, st->amg);
      if (as == HSM_OK) {
        st->amg->nu = phys->mg_sweeps == 1 ? 1 : 2;
        as = amg_tune_tail(pl, st->amg, phys->mg_tail_from, phys->mg_fused_from, phys->mg_persistent);
      }
      if (as != HSM_OK) return fail(as);
    }
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(cuda_fail(pl, e, "hsm_stepper_create"));
  *out = st;
  return HSM_OK;
}

hsm_status hsm_step(hsm_stepper st, int n_steps, double* v, double* T, double* p, int* krylov_iters) {
  if (!st) return set_error(nullptr, HSM_EINVAL, "stepper is NULL");
  if (n_steps < 0 || !v || !T || !p) return set_error(st->plan, HSM_EINVAL, "invalid step arguments");
  {
    const hsm_status ck = check_gate(st->plan);
    if (ck != HSM_OK) return ck;
  }
  bool notconv = false;
  hsm_status r = st->dim == 2 ? run_steps<2>(st, n_steps, v, T, p, krylov_iters, &notconv)
                              : run_steps<3>(st, n_steps, v, T, p, krylov_iters, &notconv);
  if (r != HSM_OK) return r;
  if (notconv) return set_error(st->plan, HSM_ENOTCONV, "a pressure solve stopped before its tolerance");
  return HSM_OK;
}

hsm_status hsm_stepper_info(hsm_stepper st, int* mg_levels, int* mg_tail_level, int* mg_tail_ctas,
                            int* mg_fused_level, int* kernels_per_iter, float* tail_ms, float* fused_ms,
                            int* mg_persistent, float* persistent_ms, int64_t* level_rows,
                            int64_t* level_entries) {
  if (!st) return set_error(nullptr, HSM_EINVAL, "stepper is NULL");
  for (int l = 0; l < kMgMaxLevels; ++l) {
    const bool in = st->amg && l < st->amg->L;
    const MgLevel* F = in ? &st->amg->lev[l] : nullptr;
    if (level_rows) level_rows[l] = in ? F->n : 0;
    if (level_entries)
      level_entries[l] = in ? F->count[0] * (int64_t)F->width[0] + F->count[1] * (int64_t)F->width[1] : 0;
  }
  if (mg_persistent) *mg_persistent = st->amg ? st->amg->persist : 0;
  if (persistent_ms) *persistent_ms = st->amg ? st->amg->persist_ms : -1.f;
  if (mg_levels) *mg_levels = st->amg ? st->amg->L : 0;
  if (mg_tail_level) *mg_tail_level = st->amg ? st->amg->lt : 0;
  if (mg_tail_ctas) *mg_tail_ctas = st->amg ? st->amg->tail_ctas : 0;
  if (mg_fused_level) *mg_fused_level = st->amg ? st->amg->lf : 0;
  if (kernels_per_iter) *kernels_per_iter = chunk_kernels(st) / chunk_iters(st) + 1;
  for (int l = 0; l < kMgMaxLevels; ++l) {
    if (tail_ms) tail_ms[l] = st->amg ? st->amg->tail_ms[l] : -1.f;
    if (fused_ms) fused_ms[l] = st->amg ? st->amg->fuse_ms[l] : -1.f;
  }
  return HSM_OK;
}

hsm_status hsm_stepper_destroy(hsm_stepper st) {
  if (!st) return HSM_OK;
  cudaStream_t s = st->plan ? st->plan->stream : nullptr;
  drop_graphs(st);
  if (st->cap) cudaStreamDestroy(st->cap);
  if (st->body) cudaStreamDestroy(st->body);
  dev_free(&st->ctl, s);
  dev_free(&st->step_iters, s);
  dev_free(&st->step_bad, s);
  if (st->amg) {
    amg_free(st->amg, s);
    delete st->amg;
    st->amg = nullptr;
  }
  dev_free(&st->wp_rbf, s);
  dev_free(&st->wn_rbf, s);
  dev_free(&st->minv, s);
  dev_free(&st->vstar, s);
  dev_free(&st->Tn, s);
  dev_free(&st->vec, s);
  dev_free(&st->hist, s);
  dev_free(&st->scal, s);
  dev_free(&st->partial, s);
  dev_free(&st->counters, s);
  dev_free(&st->gm_vec, s);
  dev_free(&st->gm_scal, s);
  dev_free(&st->gm_part, s);
  dev_free(&st->gm_cnt, s);
  cudaStreamSynchronize(s);
  delete st;
  return HSM_OK;
}

}  // extern "C"
