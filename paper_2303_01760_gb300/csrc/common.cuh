// Internal declarations shared by the translation units of libhsm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "hsm.h"

namespace hsm {

constexpr int kMaxDim = 3;
constexpr int kMaxBuildChunks = 4;  // kNN / RBF-FD solve chunks of the stencil build
constexpr int kMaxOps = 4;
constexpr int kMaxStencil = 128;
constexpr int kMaxMonomials = 84;           // C(6+3, 3): m <= 6 in 3D
constexpr int kMaxK = kMaxStencil + kMaxMonomials;
constexpr int32_t kEmpty = 0x7f7f7f7f;      // empty lattice-map slot (memset 0x7f)

// Status bits accumulated on the device while building a plan.
enum : unsigned {
  kDevSingular = 1u,   // a weight system had a zero or non-finite pivot
  kDevBounds = 2u,     // a stencil index fell outside [0, N)
  kDevKnnShort = 4u,   // fewer than n candidate nodes were found
};

struct Group {
  int width = 0;          // stencil width of the group
  int64_t count = 0;      // number of nodes in the group
  int32_t* nodes = nullptr;  // [count] node ids, ascending
  int32_t* idx = nullptr;    // [width][count] stencil node ids (index-major)
  double* w64 = nullptr;     // [nops][width][count]
  float* w32 = nullptr;      // [nops][width][count]
  int64_t w64_cap = 0;       // doubles allocated at w64 (kept across builds)
};

struct Tuning {
  int apply_threads = 256;  // threads per block of the apply kernel
  int apply_split = 1;      // lanes per RBF-FD stencil in the apply kernel (1, 2, 4)
  int rbf_lanes = 8;        // lanes per FP64 RBF-FD weight system (4, 8, 16, 32)
  int rbf_lanes32 = 8;      // lanes per FP32 + refinement weight system (4, 8, 16, 32)
  int knn_qt = 1;           // threads per kNN query (1, 2 or 4)
  // FP64 weights (arrange): 0 = MON weights beside the kNN search in the
  // stencil build graph, then one RBF-FD launch in the weights call; 1 = both
  // groups in one persistent launch with a work queue (k_weights_grouped);
  // 2 = both groups in the stencil build graph: MON beside the kNN search,
  // and the RBF-FD group in `chunks` chunks, chunk c solved on a second
  // branch while the kNN search runs on chunk c + 1
  int arrange = 0;
  int chunks = 1;  // 1, 2 or 4 (arrange 2)
  bool tuned = false;
};

struct Mlp;  // learned predictor (mlp.cu)

// Persistent workspace of the stencil build (sizes depend only on N), so the
// whole build can be replayed as one CUDA graph.
struct BuildWs {
  unsigned long long* bbox = nullptr;  // [2 * kMaxDim] ordered-bit extrema
  int* lat = nullptr;                  // [2 * kMaxDim + 5]: lattice extents, demoted, n_mon, n_rbf, flags, arrivals
  unsigned long long* bpart = nullptr; // k_bounds' per-block extrema partials
  int* lpart = nullptr;
  int32_t* ijk = nullptr;              // [dim][N]
  uint8_t* on_lat = nullptr;           // [N]
  unsigned long long* hkeys = nullptr; // lattice hash
  int32_t* hvals = nullptr;
  unsigned long long hcap = 0;
  int32_t* dmap = nullptr;             // dense lattice map, 4N + 1024 entries
  void* ldesc = nullptr;               // its extents (device)
  void* cgd = nullptr;                 // CellGrid on the device
  int32_t* cell_of = nullptr;          // [N]
  int32_t* cstart = nullptr;           // [4N + 1025]
  int32_t* ccount = nullptr;           // [4N + 1024]
  int32_t* sorted_id = nullptr;        // [N]
  double* sorted_xyz = nullptr;        // [N][kMaxDim]
  double* mon_w64 = nullptr;           // MON weights, [nops][2 dim + 1][count], room for count = N
  uint8_t* sorted_bnd = nullptr;       // [N]
  int32_t* scan_ws = nullptr;          // block sums of the cell scan
  int32_t* scan_ws2 = nullptr;         // block sums of the group partition (a parallel branch)
  int* readback = nullptr;             // pinned host: demoted, n_mon, n_rbf, flags, -, singular count, solve flags
  cudaGraphExec_t graph = nullptr;
  int graph_qt = 0;                    // kNN variant the graph was captured with
  int graph_arrange = 0;               // weights arrangement the graph was captured with
  int graph_chunks = 0;
  bool graph_timing = false;           // captured with the in-build solve's phase events
  const double* graph_w64 = nullptr;   // RBF-FD weight array and singular list the graph writes
  const int32_t* graph_sing = nullptr;
  const double* graph_spacing = nullptr;  // spacing array the graph was captured with
  int graph_kernels = 0;               // kernels per replay
  cudaStream_t cap = nullptr;
  cudaStream_t side = nullptr;         // capture branch of the MON stencils
  cudaStream_t side2 = nullptr;        // capture branch of the cell scan and scatter
  cudaStream_t side3 = nullptr;        // capture branch of the in-build RBF-FD solve (arrange 2)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_fork2 = nullptr, ev_join2 = nullptr, ev_join3 = nullptr;
  cudaEvent_t ev_chunk[kMaxBuildChunks] = {};  // kNN chunk c done
  bool ready = false;
};

}  // namespace hsm

struct hsm_plan_s {
  int dim = 2;
  int64_t N = 0;
  const double* coords = nullptr;
  const uint8_t* is_regular = nullptr;
  const uint8_t* is_boundary = nullptr;
  const double* normals = nullptr;
  const double* spacing = nullptr;  // local internodal distance [N] (NULL: h everywhere)
  double h = 0.0;
  int m = 2;
  int n = 12;
  int n_mono = 6;          // C(m+d, m)
  unsigned op_mask = 0;
  int nops = 0;
  int ops[hsm::kMaxOps] = {0, 0, 0, 0};  // operator bits in bit order
  cudaStream_t stream = nullptr;

  hsm::Group mon, rbf;
  uint8_t* kind = nullptr;      // [N] 0 = MON, 1 = RBF-FD
  int32_t* pos = nullptr;       // [N] position inside its group
  unsigned* dev_flags = nullptr;  // device status bits
  int* dev_count = nullptr;       // device counter scratch: [0] fallback list, [1] singular list
  int32_t* sing_list = nullptr;   // [2][sing_cap]: systems the FP64 solve found singular (two lists)
  int64_t sing_cap = 0;
  int64_t n_reduced = 0;          // systems solved with a lower monomial degree in the last weights call
  uint16_t* pairs = nullptr;      // [n(n-1)/2] (i << 8 | j) upper-triangle pairs
  int8_t* mono_exp = nullptr;     // [n_mono][dim] monomial exponents
  std::vector<uint16_t> h_pairs;  // host sources of the two tables (kept for the async upload)
  std::vector<int8_t> h_exp;
  int64_t n_demoted = 0;
  int64_t n_fallback = 0;
  unsigned build_flags = 0;  // device status bits of the last stencil build (MON weights included)
  int build_sing = 0;              // its in-build RBF-FD solve (arrange 2): singular systems recorded
  unsigned build_solve_flags = 0;  // and that solve's status bits
  bool stencils_built = false;
  bool weights_built = false;
  // check mode: every call that gathers through the stencils validates them
  // first (hsm_plan_set_checks, or HSM_CHECK_BOUNDS=1 at plan creation)
  bool checks = false;
  unsigned* check_flag = nullptr;  // device flag of the validation scan
  int* hrb = nullptr;              // pinned host words for the weights call's read-backs
  bool counters_fresh = false;     // the build cleared the weights call's status words
  bool rbf_from_build = false;     // the last build solved the RBF-FD weights in FP64 (arrange 2)
  hsm::Tuning tune;
  hsm_mlp mlp = nullptr;         // attached learned predictor (not owned)
  // batch validation of the learned weights: `gate_samples` stencils of the
  // batch are solved directly; when the mean relative weight error of the
  // accepted ones exceeds gate_tol, the whole batch takes the direct solve
  double gate_tol = 1e-3;
  int64_t gate_samples = 512;    // 0: no batch validation
  double gate_error = 0.0;       // of the last learned batch (-1: not measured)
  int gate_failed = 0;
  int64_t gate_accepted = 0;     // validated samples the per-stencil checks accepted
  std::string last_error;
  hsm::BuildWs ws;               // stencil-build workspace and graph
  int64_t launches = 0;          // kernels launched by this plan
  bool timing = false;
  cudaEvent_t ev[2 * HSM_PHASE_COUNT] = {};
  bool ev_used[HSM_PHASE_COUNT] = {};
};

namespace hsm {

// In check mode, validates the plan's stencils before a gathering call:
// HSM_EBOUNDS when an index lies outside its range, HSM_OK otherwise (and
// always HSM_OK outside check mode).
hsm_status check_gate(hsm_plan p);

// Event timing of one phase on the plan's stream (no-op unless enabled).
struct PhaseTimer {
  hsm_plan p;
  int ph;
  PhaseTimer(hsm_plan p_, int ph_) : p(p_), ph(ph_) {
    if (p->timing) {
      if (!p->ev[2 * ph]) {
        cudaEventCreate(&p->ev[2 * ph]);
        cudaEventCreate(&p->ev[2 * ph + 1]);
      }
      cudaEventRecord(p->ev[2 * ph], p->stream);
    }
  }
  ~PhaseTimer() {
    if (p->timing) {
      cudaEventRecord(p->ev[2 * ph + 1], p->stream);
      p->ev_used[ph] = true;
    }
  }
};

// Records a CUDA error on the plan and returns HSM_ECUDA.
hsm_status cuda_fail(hsm_plan p, cudaError_t e, const char* what);
hsm_status set_error(hsm_plan p, hsm_status s, const std::string& msg);
void set_global_error(const std::string& msg);

#define HSM_CUDA(plan, call)                                   \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return ::hsm::cuda_fail((plan), e_, #call); \
  } while (0)

template <typename T>
cudaError_t dev_alloc(T** ptr, size_t count, cudaStream_t s) {
  *ptr = nullptr;
  if (count == 0) count = 1;
  return cudaMallocAsync(reinterpret_cast<void**>(ptr), count * sizeof(T), s);
}

template <typename T>
void dev_free(T** ptr, cudaStream_t s) {
  if (*ptr) cudaFreeAsync(*ptr, s);
  *ptr = nullptr;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// ---- scan.cu -------------------------------------------------------------
// Exclusive prefix sum of in[0..n) (int32 counts) into out[0..n], out[n] = total.
// ws: scratch of scan_scratch(n) ints, or nullptr to allocate one.
// out[n] receives the total.
cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s, int32_t* ws = nullptr);
int scan_kernels(int64_t n);  // kernels one scan of n items launches
// List of indices i (ascending) with key[i] == want; count written to *count_dev.
cudaError_t select_indices(const uint8_t* key, uint8_t want, int64_t n, int32_t* out_list,
                           int32_t* out_pos, int* count_dev, cudaStream_t s, int32_t* ws = nullptr);
// Both lists of a 0/1 split in one scan: items with key == want go to
// first (in order), the others to second; pos[i] = place of i in its list;
// the list sizes go to count_first / count_second (device).
cudaError_t partition_indices(const uint8_t* key, uint8_t want, int64_t n, int32_t* first, int32_t* second,
                              int32_t* pos, int* count_first, int* count_second, cudaStream_t s, int32_t* ws);
int64_t scan_scratch(int64_t n);

// ---- stencils.cu ---------------------------------------------------------
hsm_status build_stencils(hsm_plan p);
hsm_status alloc_build_ws(hsm_plan p);
void free_build_ws(hsm_plan p);

// ---- weights.cu ----------------------------------------------------------
// MON weights enqueued inside the stencil build (count read on the device).
cudaError_t enqueue_mon_weights(hsm_plan p, const int* count_dev, double* w, cudaStream_t s);
// FP64 RBF-FD weights of chunk `chunk` of `nchunks` equal chunks of the group
// into w ([nops][n][G], G read from *G_dev on the device), on stream s; the
// stencil build enqueues one per kNN chunk.  rbf_chunk_ready sets up the
// kernel's launch shape (call it before a stream capture).
cudaError_t rbf_chunk_ready(hsm_plan p);
cudaError_t enqueue_rbf_chunk(hsm_plan p, const int* G_dev, double* w, int chunk, int nchunks, cudaStream_t s);
// FP64 weights of both stencil groups (MON and RBF-FD) in one persistent
// launch with a work queue (k_weights_grouped); MON status codes as k_mon's.
hsm_status compute_weights_grouped_fp64(hsm_plan p, uint8_t* status);
// Raises the maximum dynamic shared memory of kernel fn to at least smem
// (never lowers it: shapes cached for larger systems stay launchable).
cudaError_t raise_smem_limit(void* fn, size_t smem);
hsm_status compute_mon_weights(hsm_plan p, uint8_t* status);
hsm_status compute_rbf_weights_fp64_marked(hsm_plan p, const int32_t* list, int64_t count, uint8_t* status,
                                           uint8_t mark);
hsm_status compute_rbf_weights_fp64(hsm_plan p, const int32_t* list, int64_t count, uint8_t* status);
hsm_status compute_rbf_weights_fp32r(hsm_plan p, const int32_t* list, int64_t count, uint8_t* status,
                                     int32_t* fail_list, int* fail_count);
// FP64 solve of the listed systems with the monomials of degree <= degree
// only; solved systems get status HSM_NODE_REDUCED_DEGREE.
hsm_status compute_rbf_weights_fp64_degree(hsm_plan p, const int32_t* list, int64_t count, uint8_t* status,
                                           int degree, int32_t* sing_out);
hsm_status weights_to_f32(hsm_plan p);

// Weight systems for caller-supplied stencils, described without a plan
// (used by the allocation-free entry point in noalloc.cu).
struct RbfExternal {
  int dim = 2;
  const double* coords = nullptr;  // [dim][N]
  int64_t N = 0;
  const int32_t* idx = nullptr;    // [n][G], row 0 = stencil centres
  int64_t G = 0;
  int n = 0, n_mono = 0;
  unsigned op_mask = 0;
  int nops = 0;
  const int8_t* mono_exp = nullptr;
  const uint16_t* pairs = nullptr;
  double* w = nullptr;             // [nops][n][G]
  unsigned* flags = nullptr;
  int32_t* fail_list = nullptr;
  int* fail_count = nullptr;
  cudaStream_t stream = nullptr;
};
// Launches the FP32-refinement kernel (r32) or the FP64 kernel over the
// systems in ``list`` (nullptr = 0..count-1); no allocation.  status is
// indexed by the stencil centre; mark != 0 is written for every solved system.
cudaError_t launch_rbf_external(const RbfExternal& x, bool r32, const int32_t* list, int64_t count, uint8_t* status,
                                uint8_t mark, bool* too_big);
// Whether the FP32-refinement kernel (r32) or the FP64 kernel has a launch
// shape (shared memory per system within the block limit) for x's sizes.
cudaError_t rbf_external_fits(const RbfExternal& x, bool r32, bool* fits);

// ---- apply.cu ------------------------------------------------------------
hsm_status launch_apply(hsm_plan p, unsigned op_mask, hsm_dtype dt, const void* u, double* out,
                        cudaStream_t s);
hsm_status launch_condition(hsm_plan p, double* kappa);
hsm_status launch_wall_flux(hsm_plan p, const double* T, const int32_t* nodes, int64_t count, const double* normals,
                            double scale, double* out);

// ---- mlp.cu --------------------------------------------------------------
// Learned weights; *gate_extra receives the number of accepted stencils the
// batch validation solved directly (they carry direct-solve weights).
hsm_status compute_rbf_weights_learned(hsm_plan p, uint8_t* status, int32_t* fail_list, int* fail_count,
                                       int64_t* gate_extra);

}  // namespace hsm
