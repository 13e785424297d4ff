// Internal declarations shared by the library's translation units (not installed).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/lbm_gb300.h"

namespace lbm {

// Node flag bits in device memory.  Bits 0 and 1 are the public ones (lbm_flags).
enum : uint8_t {
  FLAG_SOLID = 1,     // solid node
  FLAG_BOUNDARY = 2,  // fluid node with at least one cut link
  FLAG_MACRO = 4,     // the step kernel stores rho, u here for the boundary pass (x_b and x_f)
};

// Model constants in the arithmetic type of a kernel (precomputed on the host so that FP32
// kernels convert nothing from FP64 at run time).
template <typename C>
struct Consts {
  C omega, one_m_omega, K;     // 1/tau, 1 - 1/tau, 3 (1 - 1/(2 tau))
  // FP64 collision coefficients per weight class c (0: axis, w = 1/9; 1: diagonal, w = 1/36):
  // w 4.5 omega, w 3 omega, w 3 K, w K; and the force weights with -G folded in: -G/3, -G/12
  C wo45[2], wo3[2], wK3[2], wK[2];
  C gw1, gw5;
  C G, psi0, rho0, a, b4, RT, two_over_G, psi_wall;
  C gx, gy, azC, azcx, azcy;
  C rho_ref;
};

// Everything a kernel needs about the model, passed by value.
struct DevParams {
  int nx, ny;
  int N;            // nx * ny
  int eos;          // lbm_eos_kind
  int scheme;       // lbm_scheme
  int has_body;     // gravity or azimuthal force present
  double tau, omega, guo_pref;  // omega = 1/tau, guo_pref = 1 - 1/(2 tau)
  double G, psi0, rho0;
  double a, b4, RT;             // Carnahan-Starling: a, b/4, R*T
  double two_over_G;
  double psi_wall;
  double gx, gy, azC, azcx, azcy;
  double rho_ref;               // 0 for FP64 storage
  Consts<double> cd;
  Consts<float> cf;
  template <typename C>
  __host__ __device__ const Consts<C>& k() const {
    if constexpr (sizeof(C) == 8) return cd; else return cf;
  }
};

// Fill cd and cf from the double fields above (host, after any change of those fields).
void finalize_consts(DevParams& p);

struct GeomCircle {
  double cx, cy, r;
  int outside;
  int pad;
};
constexpr int kMaxCircles = 16;
struct GeomParams {
  int nx, ny, N, n_circles;
  double wall_q_lo, wall_q_hi;
  GeomCircle c[kMaxCircles];
};

struct LinkRecipe;

// ---- launchers (implemented in the .cu files) ----
// geometry.cu
cudaError_t launch_geom_solid(const GeomParams& g, uint8_t* flags, cudaStream_t s);
// Counts boundary nodes and links per block; returns the per-block totals scanned in `scan`
// (int2 per block: boundary nodes, links).  Writes the grand totals into totals[0..1].
cudaError_t launch_geom_count_scan(const GeomParams& g, const uint8_t* flags, int2* block_tot,
                                   int nblocks, long long* totals, cudaStream_t s);
int geom_num_blocks(int N);
cudaError_t launch_geom_emit(const GeomParams& g, uint8_t* flags, const int2* block_off,
                             int32_t* bnode, int32_t* boff, uint8_t* ldir, double* lq,
                             cudaStream_t s);

// step.cu
// The vectorised step kernel (csrc/step_vec.cu): lattices with nx a multiple of
// step_vec_width(precision) and ny at least its tile height (8; FP16: 12).
int step_vec_width(int precision);
bool step_vec_supported(int precision, int nx, int ny);
// tma_ring (FP32 deviations, not fields_only): the two rows of the psi ring are staged by tensor
// copies instead of per-thread cp.async (tiles away from the x seam); an expired wait sets
// kErrTimeout in *err
cudaError_t launch_step_vec(int precision, const DevParams& p, const void* fa, void* fb,
                            const uint8_t* flags, double* rho_m, double* ux_m, double* uy_m,
                            bool fields_only, cudaStream_t s, bool tma_ring = false,
                            int* err = nullptr);
// path: 0 = the vectorised kernel for the deviation formats where step_vec_supported(), else
// the scalar tile kernel; 1 = the scalar tile kernel; 3 = the vectorised kernel where
// step_vec_supported() (FP64 too), its psi ring staged by cp.async only; 4 = as 0.  Paths 0 and
// 4 stage the deviation kernels' psi-ring rows by tensor copies where a tile allows (needs err)
cudaError_t launch_step(int precision, const DevParams& p, const void* fa, void* fb,
                        const uint8_t* flags, double* rho_m, double* ux_m, double* uy_m,
                        bool fields_only, cudaStream_t s, int path = 0, int* err = nullptr);

// boundary.cu
// Per-link recipe of the wall pass, fixed at creation (depends on q, tau and the scheme only):
//   f_abar(x_b, t+1) = c0 fo + c1 X1 + c2 X2 + chi rho' w_a [1 + 3 e.u_s + 4.5 (e.u_b)^2 - 1.5 u_b^2]
// with fo = B[src], X1 = L1[x1], X2 = L2[x2] (element indices, -1 = unused; bit 0 of `kind`
// selects lattice A for X2), u_s = cus u_b, or u(x_f) when uf >= 0.
struct LinkRecipe {
  int32_t* src;   // element index of the outgoing f*_a(x_b)
  int32_t* dst;   // element index of the unknown f_abar(x_b)
  int32_t* x1;
  int32_t* x2;
  int32_t* uf;    // node whose velocity is u_s (MLS, q < 1/2), or -1
  uint8_t* kind;  // bit 0: X2 from lattice A;  bit 1: ghost term present (chi != 0 path)
  double* c0;
  double* c1;
  double* c2;
  double* chi;
  double* cus;
  float* c0f;     // FP32 copies for the deviation formats
  float* c1f;
  float* c2f;
  float* chif;
  float* cusf;
};
// One lattice of a batch as the batched kernels see it.  cur and steps_left are advanced on
// the device after every step (batch_advance_kernel), so a captured graph stays valid while
// lattices join and leave the batch.
struct BatchDomain {
  DevParams p;
  void* f[2];
  const uint8_t* flags;
  double *rho_m, *ux_m, *uy_m;
  const int32_t* bnode;
  const int32_t* boff;
  const uint8_t* ldir;
  LinkRecipe recipe;
  double* carry;
  int nb;
  int cur;
  long long steps_left;
  long long steps_done;
};

size_t link_recipe_bytes(long long nl);
void link_recipe_carve(char* base, long long nl, LinkRecipe* r);
cudaError_t launch_link_setup(const DevParams& p, int nb, const int32_t* bnode,
                              const int32_t* boff, const uint8_t* ldir, const double* lq,
                              const uint8_t* flags, LinkRecipe r, cudaStream_t s);
cudaError_t launch_boundary(int precision, const DevParams& p, int nb, const int32_t* bnode,
                            const int32_t* boff, const uint8_t* ldir, LinkRecipe r,
                            const void* fa, void* fb, const double* rho_m, const double* ux_m,
                            const double* uy_m, double* carry, double* force, cudaStream_t s);
// force: per boundary node (fx, fy) of the momentum exchange with the walls, or nullptr
// Channel ends (velocity inlet at column 0, fully developed outlet at column nx - 1)
cudaError_t launch_open_x(int precision, const DevParams& p, void* fb, const uint8_t* flags,
                          double u_in, cudaStream_t s);

// batched kernels (step.cu, boundary.cu, batch.cu)
int batch_tile_rows(int ry);
int batch_tile_cols();
int batch_step_grid(int precision, int eos, int ry);
// claim: the tile counter of the claiming work queue, or nullptr for the strided one
cudaError_t launch_batch_step(int precision, int eos, int ry, const BatchDomain* doms,
                              const int4* tiles, const int* n_tiles, int* claim, int grid,
                              cudaStream_t s);
cudaError_t launch_batch_boundary(int precision, const BatchDomain* doms, const int2* items,
                                  const int* n_items, int grid, cudaStream_t s);
// persistent grid of the batch's wall pass: all the CTAs the GPU holds at once
int batch_boundary_grid(int precision);
// also resets the tile counter *claim for the next step
cudaError_t launch_batch_advance(BatchDomain* doms, int n_doms, int* claim, cudaStream_t s);

// ledger.cu
int ledger_num_blocks(int N);
// Smallest positive finite value of v[0..n) into *out (device), +inf if none.
cudaError_t launch_min_positive(const double* v, long long n, double* out, cudaStream_t s);
cudaError_t launch_mass(int precision, const DevParams& p, const void* f, const uint8_t* flags,
                        double* partials, int nblocks, double* result, int* err_flag,
                        cudaStream_t s);
cudaError_t launch_init_eq(int precision, const DevParams& p, const uint8_t* flags,
                           const double* rho, const double* ux, const double* uy, void* f,
                           cudaStream_t s);
cudaError_t launch_droplet_rho(const DevParams& p, double cx, double cy, double R, double W,
                               double rho_in, double rho_out, double* rho, double* ux, double* uy,
                               cudaStream_t s);

// step_tma.cu
bool tma_step_supported(int precision, int nx, int ny);
// one CTA waits (bounded by limit_ns) on an mbarrier that completes only with arrive; out[0]
// receives 1 if the wait saw it complete
cudaError_t launch_wait_selftest(unsigned long long limit_ns, int arrive, int* out,
                                 cudaStream_t s);
bool make_lattice_tensor_map(void* map, const void* base, int nx, int ny);
bool make_ring_tensor_map(void* map, const void* base, int nx, int ny, int box_w);
bool make_ring_tensor_maps_fp16(void* map0, void* map1, const void* base, int nx, int ny, int w0,
                                int w1);
bool make_tile_prefetch_maps(void* map0, void* map1, const void* base, int nx, int ny, int tw,
                             int vh, bool fp16);
bool make_flags_prefetch_map(void* map, const uint8_t* flags, int nx, int ny, int tw, int vh);
bool make_flags_tensor_map(void* map, const void* base, int nx, int ny);
cudaError_t launch_step_tma(const void* map, const void* flag_map, const DevParams& p,
                            const void* fa, void* fb, const uint8_t* flags, double* rho_m,
                            double* ux_m, double* uy_m, int* err, cudaStream_t s);
constexpr int kErrUnstable = 1;  // bits of the context's device error word
constexpr int kErrTimeout = 4;

// eos_host.cpp
bool cs_critical_point(double a, double b, double R, double* Tc, double* rhoc);
bool cs_maxwell(double a, double b, double R, double T, double* rho_l, double* rho_v);
double host_psi(const DevParams& p, double rho);

}  // namespace lbm

// State of one lattice (the opaque lbm_ctx of the C ABI).
struct lbm_ctx {
  lbm::DevParams p{};
  lbm::GeomParams g{};
  int precision = LBM_FP64;
  size_t lattice_bytes = 0;  // one lattice: 9 planes of nx*ny populations
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  lbm_alloc_fn alloc = nullptr;
  lbm_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  std::vector<std::pair<void*, size_t>> blocks;
  size_t device_bytes = 0;
  // device buffers
  void* f[2] = {nullptr, nullptr};
  int cur = 0;
  uint8_t* flags = nullptr;
  double *rho_m = nullptr, *ux_m = nullptr, *uy_m = nullptr;
  int32_t *bnode = nullptr, *boff = nullptr;
  uint8_t* ldir = nullptr;
  double* lq = nullptr;
  double* carry = nullptr;
  double* force = nullptr;    // per boundary node (fx, fy) of the last step's momentum exchange
  bool track_force = false;   // the wall pass fills `force` (lbm_options.track_force, inflow)
  bool open_x = false;        // channel mode (lbm_set_inflow)
  double u_in = 0.0;
  lbm::LinkRecipe recipe{};
  double* partials = nullptr;
  double* mass_out = nullptr;
  int* err_flag = nullptr;
  int2* geom_tmp = nullptr;
  long long* geom_totals = nullptr;
  int ledger_blocks = 0;
  long long nb = 0, nl = 0, n_fluid = 0;
  int64_t steps = 0;
  bool initialized = false;
  int graph_steps = 32;  // time steps per captured graph
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  double graph_rho_ref = 0.0;  // rho_ref the captured graphs hold (kernel parameters by value)
  lbm_status status = LBM_OK;
  std::string msg;
  double T = 0.0;
  bool rho_ref_auto = false;  // deviation storage: take rho_ref from the initial state
  bool use_tma = false;       // step kernel with TMA halo staging (step_tma.cu)
  int kernel_path = 0;        // lbm_options.kernel_path
  bool in_batch = false;      // owned by a batch (lbm_batch_add)
  alignas(64) unsigned char tmap[2][128];  // tensor maps of the two lattices
  alignas(64) unsigned char fmap[128];     // tensor map of the node flags
};
