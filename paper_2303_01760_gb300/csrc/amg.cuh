// Aggregation multigrid for the pressure operator of the Boussinesq step
// (Section 3: the Poisson problem of Chorin's projection), used as the right
// preconditioner of its BiCGSTAB solve.
#pragma once
#include "common.cuh"

namespace hsm {

constexpr int kMgMaxLevels = 16;
constexpr int kMgThreads = 256;
constexpr int kMgMaxRow = 64;   // distinct columns of one coarse row
constexpr int kMgCoarsest = 256;  // rows at which coarsening stops
constexpr int64_t kMgTailMaxRows = 1 << 17;  // largest level the cluster tail may start at

// One level.  Level 0 holds the nodes in the plan's two stencil groups (row =
// node id, reached through kind/pos); coarse levels hold one group whose row r
// sits at position r.  Matrices are ELL, [width][count] column-major.
struct MgLevel {
  int64_t n = 0;
  const int32_t* nodes[2] = {nullptr, nullptr};
  const int32_t* idx[2] = {nullptr, nullptr};
  const double* val[2] = {nullptr, nullptr};
  int64_t count[2] = {0, 0};
  int width[2] = {0, 0};
  int bm = 0, blocks = 0;         // blocks of group 0, all row blocks
  const uint8_t* kind = nullptr;  // level 0: group of each row
  const int32_t* pos = nullptr;   // level 0: position of each row in its group
  double* odinv = nullptr;        // omega / diagonal (0 where the diagonal vanishes)
  int32_t* agg = nullptr;         // coarse row of each row (all but the coarsest)
  int32_t* mstart = nullptr;      // rows of each coarse row: [n_coarse + 1]
  int32_t* mlist = nullptr;       // [n], ascending within each coarse row
  int cblocks = 0;                // blocks over the coarse rows
  double* f = nullptr;            // right-hand side (coarse levels)
  double* x = nullptr;
  double* y = nullptr;
  int32_t* own_idx = nullptr;     // coarse matrix storage
  double* own_val = nullptr;
};

struct Amg {
  int L = 0;
  MgLevel lev[kMgMaxLevels];
  double* binv = nullptr;  // [m][m]: leading block of the inverse of the coarsest bordered system
  int m = 0;
  double omega = 2.0 / 3.0;  // Jacobi damping
  double alpha = 1.8;        // scaling of the coarse-grid correction
  int nu = 2;                // Jacobi sweeps before and after the coarse correction (2 or 1)
  // levels lt..L-1 of a cycle run in one cluster kernel (k_mg_tail); lt = 0:
  // every level has its own kernels.  lt is picked at set-up by timing.
  int lt = 0;
  int tail_ctas = 0;             // CTAs of the tail's cluster (0: no cluster could be scheduled)
  float tail_ms[kMgMaxLevels] = {};  // 10 cycles with the tail from level l (l = 0: no tail); -1 not tried
  // levels lf.. (below the tail) use the fused down/up kernels (k_mg_down,
  // k_mg_up); lf >= L: none.  Picked with lt by timing.
  int lf = kMgMaxLevels;
  float fuse_ms[kMgMaxLevels] = {};  // 10 cycles, no tail, fused from level l; -1 not tried
  MgLevel* dlev = nullptr;       // device copy of lev[0..L)
  // persist = 1: the whole cycle runs as one cooperative kernel (k_mg_cycle)
  // of pblocks x kMgCycleThreads threads, its phases separated by a
  // grid-wide barrier on gbar ([0] arrivals, [1] generation, [2] timeout
  // flag).  Picked by timing against the best of the shapes above.
  int persist = 0;
  int pblocks = 0;
  unsigned* gbar = nullptr;
  float persist_ms = -1.f;        // 10 cycles of k_mg_cycle; -1 not tried
};

constexpr int kMgCycleThreads = 512;

// Builds the hierarchy of the pressure operator whose rows are the plan's
// stencils with weights wp_mon ([mon.width][mon.count]) and wp_rbf
// ([rbf.width][rbf.count]); the centre is the first entry of every stencil.
hsm_status amg_setup(hsm_plan pl, const double* wp_mon, const double* wp_rbf, double alpha, Amg* amg);
// Enqueues one V(2,2)-cycle on s: out[0..N) = M^-1 in[0..N), out[N] = in[N]
// (the border unknown of the bordered system is left as it is).  Every kernel
// returns at once when *done != 0; done = nullptr runs the cycle unconditionally
// (inside a device-side loop that ends on convergence by itself).
cudaError_t amg_vcycle(const Amg& amg, const double* in, double* out, const double* done, cudaStream_t s);
int amg_kernels_per_cycle(const Amg& amg);
// Picks the first level of the cluster tail (or none) and the first level of
// the fused down/up kernels (or none) by timing a few cycles of each choice
// on scratch vectors of N + 1 entries.  Synchronises.
// tail_from / fused_from / persistent as hsm_phys.mg_tail_from /
// mg_fused_from / mg_persistent (0: time).
hsm_status amg_tune_tail(hsm_plan pl, Amg* amg, int tail_from, int fused_from, int persistent);
// Clears the grid barrier of the cooperative cycle (arrivals, generation,
// timeout flag); enqueued on s.  No-op for the other shapes.
cudaError_t amg_reset_barrier(const Amg& amg, cudaStream_t s);
// Device address of the barrier's timeout flag (nullptr for the other shapes).
const unsigned* amg_timeout_flag(const Amg& amg);
void amg_free(Amg* amg, cudaStream_t s);

}  // namespace hsm
