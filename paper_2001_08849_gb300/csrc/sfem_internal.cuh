// Internal declarations of the FS-FEM-T4 CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <memory>
#include <string>
#include <vector>

#include "../../include/sfem.h"
#include "coarse.cuh"

namespace sfem {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
struct Error {
  int status;
  std::string msg;
};

void set_last_error(const std::string &msg);

#define SFEM_CUDA(call)                                                               \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      throw ::sfem::Error{SFEM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_) + \
                                          " (" + __FILE__ + ":" + std::to_string(__LINE__) + ")"}; \
  } while (0)

// kernel-launch accounting (sfem_launch_count); launches recorded during a
// stream capture are not counted, graph launches add their node count
void count_launches(int64_t n);
bool capturing();
void set_capturing(bool on);

#define SFEM_CHECK_LAUNCH()                        \
  do {                                             \
    SFEM_CUDA(cudaGetLastError());                 \
    if (!::sfem::capturing()) ::sfem::count_launches(1); \
  } while (0)

#define SFEM_REQUIRE(cond, code, text)                       \
  do {                                                       \
    if (!(cond)) throw ::sfem::Error{(code), std::string(text)}; \
  } while (0)

// ---------------------------------------------------------------------------
// device status word written by setup kernels (no traps: counters only)
// ---------------------------------------------------------------------------
struct DevStatus {
  unsigned long long bad_index;       // node id out of range
  unsigned long long bad_tets;        // degenerate or non-finite tets
  unsigned long long slivers;         // quality < 1e-3
  unsigned long long bad_faces;       // face with more than two tets
  unsigned long long too_many_inc;    // node in more than kMaxInc tets
  unsigned long long max_inc;         // largest node->tet incidence
  unsigned long long bad_dir;         // Dirichlet DOF out of range
  unsigned long long bad_tri;         // traction triangle node out of range
  unsigned long long minq_bits;       // min quality, as ordered bits of a double
  unsigned long long minv_bits;       // min volume
  unsigned long long maxv_bits;       // max volume
};

// Largest node->tet incidence handled by the adjacency kernels.
constexpr int kMaxInc = 128;

// Solver scalars, kept on the device for the whole solve so that no
// iteration needs a host round trip.
struct SolveScalars {
  double rz, rz_prev, pq, rr, alpha, beta;
  double bb;        // ||r||^2 at the last (re)start
  double tol2;      // squared stopping threshold on ||r||^2
  double rmax2;     // largest ||r||^2 since the last reliable update
  double delta2;    // reliable-update trigger: ||r||^2 < delta2 * rmax2 (0: never)
  int done;         // 1: stop the captured iterations; kernels become no-ops
  int status;       // 0 ok, 1 breakdown
  int iter;         // completed iterations
  int max_iter;
  int reason;       // why done: 1 converged, 2 reliable update due, 3 iteration cap
  int pad[3];
  double rzj, rzc;  // two-level iterations: z.r = r.D^-1 r (update pass) + rc.C rc (coarse product)
};

// ---------------------------------------------------------------------------
// allocator
// ---------------------------------------------------------------------------
struct Allocator {
  sfem_alloc_fn alloc = nullptr;
  sfem_free_fn free = nullptr;
  void *user = nullptr;
  cudaStream_t stream = nullptr;
  struct Block {
    void *p;
    size_t n;
  };
  std::vector<Block> blocks;

  void *raw(size_t bytes);
  void drop(void *p);  // free one block early (temporaries)
  void release_all();
  template <class T>
  T *get(size_t n) {
    return static_cast<T *>(raw(n * sizeof(T)));
  }
};

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct Csr {
  int64_t n_rows = 0, nnz = 0;
  int64_t *row_ptr = nullptr;
  int32_t *col = nullptr;
  double *val = nullptr;
  // node-level adjacency (pattern of 3x3 blocks)
  int64_t *nptr = nullptr;   // n_nodes + 1
  int32_t *nadj = nullptr;   // nptr[n_nodes]
};

// tiled single-pass FP32 operator (tiles.cu)
struct TileData {
  bool ready = false;
  int64_t n_tiles = 0, total_halo = 0, total_nodes = 0;
  int32_t *perm = nullptr;       // tile order -> input tet id
  int32_t *iperm = nullptr;      // input tet id -> tile order
  int32_t *tile_start = nullptr; // n_tiles + 1, ranges of tile-order tets
  int64_t *hoff = nullptr;       // n_tiles + 1 halo offsets
  int64_t *noff = nullptr;       // n_tiles + 1 node-list offsets
  int32_t *halo_tet = nullptr;   // halo tets (tile order)
  uint2 *halo_lconn = nullptr;   // their local connectivity (4 x 16 bit)
  int32_t *tile_nodes = nullptr; // node ids per tile, in the order of the slot layout
  uint32_t *node_inc = nullptr;  // per tile node: base of its slot group | own-slot count << 16
  float4 *rec = nullptr;         // 64-byte per-tet records (tile order): V_e grad N_1..3,
                                 // V_e, local connectivity, local neighbours, slot positions
  int max_halo = 0, max_nodes = 0;
  int slot_stride = 0;           // floats per component array of a tile's force slots
  // persistent prefetching form of the operator (tiles.cu): shared-memory
  // layout, grid, and a device word set when one of its waits gave up
  int pf_capN = 0, pf_capH = 0, pf_capH2 = 0, pf_capR = 0, pf_ibytes = 0, pf_off_i = 0, pf_off_h = 0,
      pf_off_u = 0;
  int pf_off_w[2] = {0, 0};      // [0] FP32 input, [1] FP64 input
  size_t pf_smem[2] = {0, 0};
  int pf_grid[2] = {0, 0};       // 0: the one-CTA-per-tile form is used
  int pf_threads[2] = {0, 0};    // threads per CTA of the persistent form (256 or 512)
  int *err = nullptr;
  size_t smem = 0;               // dynamic shared memory of the operator kernel
};

// regular grid of patches over a bounding box (learned correction and
// coarse space)
struct PatchGrid {
  int d[3];
  double lo[3], ext[3];
};

// two-level preconditioner data (coarse.cu); device arrays owned by the
// context's allocator
struct Coarse {
  PatchGrid g{};
  CoarseDev dev{};
  int probes = 0;
  bool fp64_factor = false;  // the FP32 Cholesky of A_c broke down
  double setup_ms = 0.0;
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  Allocator mem;

  int64_t n_nodes = 0, n_tets = 0, ndof = 0, n_faces = 0, n_int = 0, n_bnd = 0;
  int64_t n_dir = 0, n_tri = 0;
  int nrhs = 1;
  double E = 0, nu = 0, lam = 0, mu = 0;

  // inputs (device copies)
  double *xyz = nullptr;      // n_nodes*3
  int32_t *tets = nullptr;    // n_tets*4 (int4-aligned)
  int32_t *dir_dofs = nullptr;
  double *dir_vals = nullptr;

  // FP64 geometry
  double *vol = nullptr;      // n_tets
  double *grad = nullptr;     // n_tets*12: grad N_0..3 (x,y,z)

  // topology
  int64_t *n2t_ptr = nullptr; // n_nodes + 1
  int32_t *n2t = nullptr;     // 4*n_tets, tets of each node ascending
  int32_t *nbr = nullptr;     // n_tets*4: tet across the face opposite vertex a, -1
  int32_t *nbr_slot = nullptr;// n_tets*4: local vertex of nbr not on that face
  int32_t *face_tet = nullptr;// n_faces*2
  int32_t *face_slot = nullptr;// n_faces*2
  double *Vk = nullptr;       // n_faces

  // matrix-free operator data: Gs = V_e grad N_1..3 (planar, 9 x n_tets),
  // kap[e][a] = 1/(4 (V_e + V_nbr)) or 1/(4 V_e) on exterior faces.
  double *Gs64 = nullptr;
  double *kap64 = nullptr;    // n_tets*4
  float *Gs32 = nullptr;
  float *kap32 = nullptr;     // n_tets*4

  // boundary conditions and loads
  uint8_t *dmask = nullptr;   // ndof: 1 free, 0 prescribed
  double *g = nullptr;        // ndof prescribed values (0 elsewhere)
  double *f = nullptr;        // nrhs*ndof traction loads
  double *diag = nullptr;     // ndof diagonal of K
  double *dinv64 = nullptr;   // ndof: P/diag (0 on prescribed DOFs)
  float *dinv32 = nullptr;
  std::vector<double> bnorm;  // ||b|| per rhs

  Csr csr;
  bool assembled = false;
  TileData tl;
  double bbox_lo[3] = {0, 0, 0}, bbox_hi[3] = {0, 0, 0};  // node bounding box (set with the tiles)

  DevStatus *dstat = nullptr;
  DevStatus hstat{};
  double setup_ms = 0;

  // scratch for the operators and reductions
  void *w_scratch = nullptr;     // per-tet strains (8 values per tet per rhs)
  double *ns_sig = nullptr;      // NS-FEM: nodal stresses (6 per node), allocated on first use
  // ES-FEM (built on first use): edge ids of every tet (6 per tet), edge
  // domain volumes, per-edge strain / stress accumulators (6 per edge)
  int32_t *es_te = nullptr;
  double *es_Vk = nullptr, *es_acc = nullptr;
  int64_t n_edges = 0;
  size_t w_bytes = 0;
  double *red_partial = nullptr; // per-block partial sums
  int red_blocks = 0;
  unsigned int *tickets = nullptr; // zeroed ticket counters of grid reductions
  SolveScalars *scal = nullptr;
  SolveScalars *h_scal = nullptr; // pinned host copies (2 slots), allocated on first chunked solve
  bool g_zero = true;             // all prescribed displacements are zero
  cudaStream_t cap_stream = nullptr; // private stream used only for graph capture
  std::shared_ptr<Coarse> coarse;    // two-level preconditioner, if set up
};

// ---------------------------------------------------------------------------
// helpers shared between translation units
// ---------------------------------------------------------------------------
inline int grid_for(int64_t n, int block) { return (int)((n + block - 1) / block); }

// exclusive scan of n int32 counts into out[0..n] (int64); returns out[n]
int64_t scan_counts(Ctx &c, const int32_t *counts, int64_t n, int64_t *out);

// operators (operator.cu): raw K u (no masking) for nrhs vectors
void apply_mf64(Ctx &c, const double *u, double *y, int nrhs, double *energy_partial);
void apply_mf32(Ctx &c, const float *u, float *y, int nrhs, double *energy_partial);
void apply_csr64(Ctx &c, const double *u, double *y, int nrhs, const double *dotv,
                 double *dot_partial);
void ensure_w_scratch(Ctx &c, size_t bytes);
// NS-FEM-T4 operator (nsfem.cu): y += K_NS u, energy += u^T K_NS u (may be
// null); apply_ns64 zeroes y first
void launch_ns64(Ctx &c, cudaStream_t st, const double *u, double *y, double *energy, const int *done);
void apply_ns64(Ctx &c, const double *u, double *y);
// ES-FEM-T4 operator (esfem.cu): prepare_es64 builds the edge table (before
// any stream capture); launch_es64 as launch_ns64; apply_es64 zeroes y first
void prepare_es64(Ctx &c);
void launch_es64(Ctx &c, cudaStream_t st, const double *u, double *y, double *energy, const int *done);
void apply_es64(Ctx &c, const double *u, double *y);
// stream-explicit launchers used inside captured solver iterations; kernels
// return immediately when *done != 0
// T: geometry and arithmetic type; TU / TY: input / output vector types
template <class T, class TU>
void launch_mf_strain(Ctx &c, cudaStream_t st, const T *Gs, const TU *u, int nrhs, T *w, const int *done);
template <class T, class TY>
void launch_mf_stress(Ctx &c, cudaStream_t st, const T *Gs, const T *kap, const T *w, TY *y, int nrhs,
                      double *energy_out, const int *done);
void launch_csr64(Ctx &c, cudaStream_t st, const double *u, double *y, const double *dotv, double *dot_out,
                  const int *done);
int reduction_blocks();
// sum of squares of x[0..n) on the device, FP64 accumulation (synchronises)
double device_norm2(Ctx &c, const double *x, int64_t n);

// setup pieces used by other units
void compute_diag(Ctx &c);
void build_tiles(Ctx &c);
// throws SFEM_ECUDA if a wait of the prefetching tiled operator gave up
void check_tile_error(Ctx &c);
// tiled FP32 operator y += K u (y must be zeroed by the caller); u, y of
// type TU/TY (float or double); the energy u^T K u is added to *energy_out
// (zeroed by the caller)
template <class TU, class TY>
void launch_mf32_tiled(Ctx &c, cudaStream_t st, const TU *u, TY *y, double *energy_out, const int *done);

// coarse correction of the two-level preconditioner (coarse.cu), on
// stream st, all returning at once while *done != 0:
// rc = Pi^T r (r masked), then yc = C rc
void coarse_correction(Ctx &c, cudaStream_t st, const double *r, const int *done);
void coarse_correction(Ctx &c, cudaStream_t st, const float *r, const int *done);
// the context's coarse space, built if missing: patches of patch_nodes node
// spacings (0: the default options; the default options again if that
// setup fails); false when none can be built
bool ensure_coarse(Ctx &c, int patch_nodes = 0);
// yc = C rc only (the fused two-level iterations restrict r themselves)
// (with rzc: rc.C rc added to *rzc)
void coarse_gemv(const CoarseDev &cs, cudaStream_t st, const int *done, double *rzc = nullptr);
// rc = Pi^T r only (fixed order; yc zeroed)
void coarse_restrict(Ctx &c, cudaStream_t st, const double *r, const int *done);

// solves (solve.cu); a Snapshot, when given, sees the iterate x and the
// residual r (device, ndof) of the flexible PCG before its first iteration
// and after every chunk of check_every iterations
using Snapshot = std::function<void(const double *x, const double *r, int iter)>;
// row collection and direction window of the truncated flexible CG with the
// learned coarse solve (cnet.cu)
struct CnRunArgs {
  int window = 0;       // directions kept (0: 5)
  int snap_every = 0;   // a training row every this many iterations (0: none)
  float *X = nullptr, *T = nullptr;  // rows x n_coarse each (device)
  int64_t cap = 0;      // rows the buffers hold
  int64_t rows = 0;     // rows already there on entry, total on return
};
void solve_impl(Ctx &c, const double *f_extra, double *u, const sfem_solve_opts &o, sfem_solve_info &info,
                const Snapshot *snap = nullptr, CnRunArgs *cn = nullptr);
// truncated flexible CG with the learned coarse solve `model` (NULL: the
// Jacobi preconditioner alone); same contract as solve_fpcg
void solve_cnet(Ctx &c, const void *model, CnRunArgs *args, int op64, double *x, double *r, double bnorm,
                double tol, int max_iter, sfem_solve_info &info, const std::function<double()> &true_residual);
// flexible PCG with the learned correction (learned.cu); r holds the masked
// residual of x on entry; true_residual() recomputes it and returns ||r||/||b||
void solve_fpcg(Ctx &c, const void *learned, int op64, double *x, double *r, double bnorm, double tol, int max_iter,
                int chunk, int window, int pace, sfem_solve_info &info, const std::function<double()> &true_residual,
                const Snapshot *snap);

}  // namespace sfem

// opaque handle of the ABI
struct sfem_ctx {
  sfem::Ctx c;
};
