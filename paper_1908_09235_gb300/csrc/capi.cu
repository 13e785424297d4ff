// C ABI of the library (declared in include/lbm_gb300.h): argument checks, device memory,
// geometry set-up, the time-step loop (CUDA graphs of whole steps) and field transfer.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbm_internal.h"

using namespace lbm;

namespace {
constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
}  // namespace


namespace {

lbm_status fail(lbm_ctx* c, lbm_status s, const std::string& m) {
  if (c && c->status == LBM_OK) {
    c->status = s;
    c->msg = m;
  }
  return s;
}

lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* where) {
  return fail(c, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA(ctx, call)                                   \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
  } while (0)

void* dev_alloc(lbm_ctx* c, size_t bytes) {
  void* ptr = nullptr;
  if (c->alloc) {
    ptr = c->alloc(bytes, c->alloc_user);
  } else if (cudaMallocAsync(&ptr, bytes, c->stream) != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
  }
  if (ptr) {
    c->blocks.emplace_back(ptr, bytes);
    c->device_bytes += bytes;
  }
  return ptr;
}

void release_all(lbm_ctx* c) {
  for (int k = 0; k < 2; ++k)
    if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
  if (c->stream || true) cudaStreamSynchronize(c->stream);
  for (auto& b : c->blocks) {
    if (c->free_fn)
      c->free_fn(b.first, c->alloc_user);
    else
      cudaFreeAsync(b.first, c->stream);
  }
  c->blocks.clear();
  if (!c->free_fn) cudaStreamSynchronize(c->stream);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
}

// Carve sub-buffers out of one allocation.
struct Carver {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base + off);
    off += align_up(count * sizeof(T));
    return p;
  }
};

cudaError_t launch_bulk(lbm_ctx* c, cudaStream_t s, int cur) {
  if (c->use_tma)
    return launch_step_tma(c->tmap[cur], c->fmap, c->p, c->f[cur], c->f[1 - cur], c->flags,
                           c->rho_m, c->ux_m, c->uy_m, c->err_flag, s);
  return launch_step(c->precision, c->p, c->f[cur], c->f[1 - cur], c->flags, c->rho_m, c->ux_m,
                     c->uy_m, false, s, c->kernel_path, c->err_flag);
}

lbm_status launch_one_step(lbm_ctx* c, cudaStream_t s, int cur) {
  const void* fa = c->f[cur];
  void* fb = c->f[1 - cur];
  cudaError_t e = launch_bulk(c, s, cur);
  if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
  e = launch_boundary(c->precision, c->p, (int)c->nb, c->bnode, c->boff, c->ldir, c->recipe, fa,
                      fb, c->rho_m, c->ux_m, c->uy_m, c->carry,
                      c->track_force ? c->force : nullptr, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "boundary kernel launch");
  if (c->open_x) {
    e = launch_open_x(c->precision, c->p, fb, c->flags, c->u_in, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "channel-end kernel launch");
  }
  return LBM_OK;
}

lbm_status build_graph(lbm_ctx* c, int parity) {
  cudaGraph_t graph = nullptr;
  LBM_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  int cur = parity;
  lbm_status st = LBM_OK;
  for (int k = 0; k < c->graph_steps && st == LBM_OK; ++k) {
    st = launch_one_step(c, c->cap_stream, cur);
    cur = 1 - cur;
  }
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
  if (st != LBM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&c->graph[parity], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
  c->graph_rho_ref = c->p.rho_ref;
  return LBM_OK;
}

bool is_fin(double v) { return std::isfinite(v); }

}  // namespace

extern "C" {

const char* lbm_status_string(lbm_status s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of device memory";
    case LBM_ECUDA: return "CUDA error";
    case LBM_EUNSTABLE: return "unstable: non-positive or non-finite density";
    case LBM_ETIMEOUT: return "device wait timed out";
    case LBM_ESTATE: return "call out of order";
  }
  return "unknown status";
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->msg.c_str() : "null context"; }

lbm_status lbm_coexistence(const lbm_eos* eos, double* rho_l, double* rho_v) {
  if (!eos || !rho_l || !rho_v || eos->kind != LBM_EOS_CS) return LBM_EINVAL;
  double Tc, rhoc;
  if (!cs_critical_point(eos->a, eos->b, eos->R, &Tc, &rhoc)) return LBM_EINVAL;
  if (!(eos->T_over_Tc > 0.0 && eos->T_over_Tc < 1.0)) return LBM_EINVAL;
  if (!cs_maxwell(eos->a, eos->b, eos->R, eos->T_over_Tc * Tc, rho_l, rho_v)) return LBM_EINVAL;
  return LBM_OK;
}

lbm_status lbm_create(const lbm_geometry* geo, const lbm_eos* eos, double tau, int32_t scheme,
                      const lbm_options* opt, lbm_ctx** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (!geo || !eos) return LBM_EINVAL;
  if (geo->nx < 4 || geo->ny < 4 || geo->nx > 65536 || geo->ny > 65536) return LBM_EINVAL;
  if (9LL * geo->nx * geo->ny >= (1LL << 31)) return LBM_EINVAL;  // 32-bit element offsets
  if (geo->n_circles < 0 || geo->n_circles > kMaxCircles) return LBM_EINVAL;
  if (geo->n_circles > 0 && !geo->circles) return LBM_EINVAL;
  if (!(tau > 0.5) || !is_fin(tau)) return LBM_EINVAL;
  if (scheme < LBM_HBB || scheme > LBM_BOUZIDI_L_A) return LBM_EINVAL;
  if (scheme == LBM_FH && std::fabs(tau - 1.0) < 1e-3) return LBM_EINVAL;  // chi of Eq. (9)
  if (eos->kind < LBM_EOS_NONE || eos->kind > LBM_EOS_CS) return LBM_EINVAL;
  const int precision = opt ? opt->precision : LBM_FP64;
  if (precision != LBM_FP64 && precision != LBM_FP32_DEV && precision != LBM_FP16_DEV)
    return LBM_EINVAL;
  if (opt && ((opt->alloc == nullptr) != (opt->free == nullptr))) return LBM_EINVAL;
  if (opt && opt->graph_steps < 0) return LBM_EINVAL;
  for (int k = 0; k < geo->n_circles; ++k) {
    const lbm_circle& cc = geo->circles[k];
    if (!(cc.r > 0) || !is_fin(cc.cx) || !is_fin(cc.cy) || !is_fin(cc.r)) return LBM_EINVAL;
    if (cc.cx - cc.r - 2 < 0 || cc.cx + cc.r + 2 > geo->nx - 1 || cc.cy - cc.r - 2 < 0 ||
        cc.cy + cc.r + 2 > geo->ny - 1)
      if (!cc.solid_outside) return LBM_EINVAL;  // would cross the periodic seam
  }
  if (!(geo->wall_q_lo <= 1.0) || !(geo->wall_q_hi <= 1.0)) return LBM_EINVAL;

  lbm_ctx* c = new lbm_ctx();
  c->precision = precision;
  {
    const size_t nn = (size_t)geo->nx * geo->ny;
    // FP16: rest population as FP32, the eight moving ones as FP16
    c->lattice_bytes = precision == LBM_FP64 ? 72 * nn : (precision == LBM_FP32_DEV ? 36 * nn : 20 * nn);
  }
  c->stream = opt ? (cudaStream_t)opt->stream : nullptr;
  if (opt && opt->alloc) {
    c->alloc = opt->alloc;
    c->free_fn = opt->free;
    c->alloc_user = opt->alloc_user;
  }
  if (opt && opt->graph_steps > 0) c->graph_steps = opt->graph_steps + (opt->graph_steps & 1);

  DevParams& p = c->p;
  p.nx = geo->nx;
  p.ny = geo->ny;
  p.N = geo->nx * geo->ny;
  p.eos = eos->kind;
  p.scheme = scheme;
  p.tau = tau;
  p.omega = 1.0 / tau;
  p.guo_pref = 1.0 - 1.0 / (2.0 * tau);
  p.G = eos->G;
  p.psi0 = eos->psi0;
  p.rho0 = eos->rho0;
  p.gx = eos->gx;
  p.gy = eos->gy;
  p.azC = eos->azim_C;
  p.azcx = eos->azim_cx;
  p.azcy = eos->azim_cy;
  p.has_body = (eos->gx != 0.0 || eos->gy != 0.0 || eos->azim_C != 0.0) ? 1 : 0;
  p.rho_ref = precision == LBM_FP64 ? 0.0 : ((opt && opt->rho_ref > 0) ? opt->rho_ref : 1.0);
  c->rho_ref_auto = precision != LBM_FP64 && !(opt && opt->rho_ref > 0);
  if (eos->kind == LBM_EOS_CS) {
    double Tc, rhoc;
    if (!(eos->G < 0) || !cs_critical_point(eos->a, eos->b, eos->R, &Tc, &rhoc) ||
        !(eos->T_over_Tc > 0)) {
      delete c;
      return LBM_EINVAL;
    }
    c->T = eos->T_over_Tc * Tc;
    p.a = eos->a;
    p.b4 = eos->b / 4.0;
    p.RT = eos->R * c->T;
  }
  if (eos->kind != LBM_EOS_NONE && eos->G == 0.0) {
    delete c;
    return LBM_EINVAL;
  }
  if (eos->kind == LBM_EOS_EXP && !(eos->rho0 > 0)) {
    delete c;
    return LBM_EINVAL;
  }
  p.two_over_G = eos->kind != LBM_EOS_NONE ? 2.0 / eos->G : 0.0;
  p.psi_wall = eos->kind != LBM_EOS_NONE ? host_psi(p, eos->rho_wall) : 0.0;
  finalize_consts(p);

  GeomParams& g = c->g;
  g.nx = geo->nx;
  g.ny = geo->ny;
  g.N = p.N;
  g.n_circles = geo->n_circles;
  g.wall_q_lo = geo->wall_q_lo;
  g.wall_q_hi = geo->wall_q_hi;
  for (int k = 0; k < geo->n_circles; ++k)
    g.c[k] = GeomCircle{geo->circles[k].cx, geo->circles[k].cy, geo->circles[k].r,
                        geo->circles[k].solid_outside ? 1 : 0, 0};

  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return LBM_ECUDA;
  }

  // ---- first allocation: lattices, flags, macro arrays, ledger and scan scratch ----
  const size_t N = (size_t)p.N;
  const int gblocks = geom_num_blocks(p.N);
  c->ledger_blocks = ledger_num_blocks(p.N);
  size_t bytes = 2 * align_up(c->lattice_bytes) + align_up((N + 3) / 4 * 4) +
                 3 * align_up(N * 8) + align_up(c->ledger_blocks * 8) + align_up(8) +
                 align_up(sizeof(int)) + align_up(gblocks * sizeof(int2)) + align_up(16);
  void* base = dev_alloc(c, bytes);
  if (!base) {
    release_all(c);
    delete c;
    return LBM_ENOMEM;
  }
  Carver cv{(char*)base};
  c->f[0] = cv.take<char>(c->lattice_bytes);
  c->f[1] = cv.take<char>(c->lattice_bytes);
  c->flags = cv.take<uint8_t>((N + 3) / 4 * 4);
  c->rho_m = cv.take<double>(N);
  c->ux_m = cv.take<double>(N);
  c->uy_m = cv.take<double>(N);
  c->partials = cv.take<double>(c->ledger_blocks);
  c->mass_out = cv.take<double>(1);
  c->err_flag = cv.take<int>(1);
  c->geom_tmp = cv.take<int2>(gblocks);
  c->geom_totals = cv.take<long long>(2);

  auto bail = [&](cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    release_all(c);
    delete c;
    std::fprintf(stderr, "lbm_create: %s\n", m.c_str());
    return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
  };
  cudaError_t e;
  if ((e = cudaMemsetAsync(c->flags, 0, (N + 3) / 4 * 4, c->stream)) != cudaSuccess)
    return bail(e, "memset flags");
  if ((e = cudaMemsetAsync(c->err_flag, 0, sizeof(int), c->stream)) != cudaSuccess)
    return bail(e, "memset err");
  if ((e = launch_geom_solid(g, c->flags, c->stream)) != cudaSuccess) return bail(e, "geom solid");
  if ((e = launch_geom_count_scan(g, c->flags, c->geom_tmp, gblocks, c->geom_totals, c->stream)) !=
      cudaSuccess)
    return bail(e, "geom count");
  long long tot[2] = {0, 0};
  if ((e = cudaMemcpyAsync(tot, c->geom_totals, sizeof(tot), cudaMemcpyDeviceToHost, c->stream)) !=
      cudaSuccess)
    return bail(e, "copy totals");
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(e, "sync");
  c->nb = tot[0];
  c->nl = tot[1];

  // ---- second allocation: boundary-link CSR and the FP64 rounding carry ----
  if (c->nb > 0) {
    size_t b2 = align_up(c->nb * 4) + align_up((c->nb + 1) * 4) + align_up(c->nl) +
                align_up(c->nl * 8) + align_up(c->nb * 8) + align_up(c->nb * 16) +
                align_up(link_recipe_bytes(c->nl));
    void* base2 = dev_alloc(c, b2);
    if (!base2) {
      release_all(c);
      delete c;
      return LBM_ENOMEM;
    }
    Carver c2{(char*)base2};
    c->bnode = c2.take<int32_t>(c->nb);
    c->boff = c2.take<int32_t>(c->nb + 1);
    c->ldir = c2.take<uint8_t>(c->nl);
    c->lq = c2.take<double>(c->nl);
    c->carry = c2.take<double>(c->nb);
    c->force = c2.take<double>(2 * c->nb);
    link_recipe_carve(c2.take<char>(link_recipe_bytes(c->nl)), c->nl, &c->recipe);
    if ((e = launch_geom_emit(g, c->flags, c->geom_tmp, c->bnode, c->boff, c->ldir, c->lq,
                              c->stream)) != cudaSuccess)
      return bail(e, "geom emit");
    int32_t last = (int32_t)c->nl;
    if ((e = cudaMemcpyAsync(c->boff + c->nb, &last, 4, cudaMemcpyHostToDevice, c->stream)) !=
        cudaSuccess)
      return bail(e, "copy boff");
    if ((e = cudaMemsetAsync(c->carry, 0, c->nb * 8, c->stream)) != cudaSuccess)
      return bail(e, "memset carry");
    if ((e = cudaMemsetAsync(c->force, 0, c->nb * 16, c->stream)) != cudaSuccess)
      return bail(e, "memset force");
    if ((e = launch_link_setup(c->p, (int)c->nb, c->bnode, c->boff, c->ldir, c->lq, c->flags,
                               c->recipe, c->stream)) != cudaSuccess)
      return bail(e, "link setup");
  }
  // fluid node count (host, once)
  std::vector<uint8_t> hf(N);
  if ((e = cudaMemcpyAsync(hf.data(), c->flags, N, cudaMemcpyDeviceToHost, c->stream)) !=
      cudaSuccess)
    return bail(e, "copy flags");
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(e, "sync");
  long long nf = 0;
  for (size_t k = 0; k < N; ++k) nf += (hf[k] & FLAG_SOLID) ? 0 : 1;
  c->n_fluid = nf;
  if ((e = cudaMemsetAsync(c->f[0], 0, c->lattice_bytes, c->stream)) != cudaSuccess)
    return bail(e, "memset f0");
  if ((e = cudaMemsetAsync(c->f[1], 0, c->lattice_bytes, c->stream)) != cudaSuccess)
    return bail(e, "memset f1");
  c->kernel_path = opt ? opt->kernel_path : 0;
  c->track_force = opt && opt->track_force != 0;
  if (opt && opt->kernel_path == 2 && tma_step_supported(precision, geo->nx, geo->ny))
    c->use_tma = make_lattice_tensor_map(c->tmap[0], c->f[0], geo->nx, geo->ny) &&
                 make_lattice_tensor_map(c->tmap[1], c->f[1], geo->nx, geo->ny) &&
                 make_flags_tensor_map(c->fmap, c->flags, geo->nx, geo->ny);
  *out = c;
  return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  release_all(c);
  delete c;
}

static lbm_status init_common(lbm_ctx* c) {
  // captured steps hold the kernel parameters by value: keep them while rho_ref is unchanged
  if (c->p.rho_ref != c->graph_rho_ref)
    for (int k = 0; k < 2; ++k)
      if (c->graph[k]) {
        cudaGraphExecDestroy(c->graph[k]);
        c->graph[k] = nullptr;
      }
  LBM_CUDA(c, launch_init_eq(c->precision, c->p, c->flags, c->rho_m, c->ux_m, c->uy_m, c->f[0],
                             c->stream));
  LBM_CUDA(c, cudaMemsetAsync(c->f[1], 0, c->lattice_bytes, c->stream));
  if (c->nb > 0) LBM_CUDA(c, cudaMemsetAsync(c->carry, 0, c->nb * 8, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  c->cur = 0;
  c->steps = 0;
  c->initialized = true;
  return LBM_OK;
}

lbm_status lbm_init_fields(lbm_ctx* c, const double* rho, const double* ux, const double* uy) {
  if (!c) return LBM_EINVAL;
  if (c->status) return c->status;
  if (!rho) return LBM_EINVAL;
  const size_t N = (size_t)c->p.N;
  LBM_CUDA(c, cudaMemcpyAsync(c->rho_m, rho, N * 8, cudaMemcpyHostToDevice, c->stream));
  if (c->rho_ref_auto) {  // smallest positive finite initial density, found on the device
    // (mass_out is free scratch outside lbm_mass)
    LBM_CUDA(c, launch_min_positive(c->rho_m, (long long)N, c->mass_out, c->stream));
    double m = 0.0;
    LBM_CUDA(c, cudaMemcpyAsync(&m, c->mass_out, 8, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (std::isfinite(m) && m > 0) c->p.rho_ref = m;
    finalize_consts(c->p);
  }
  if (ux)
    LBM_CUDA(c, cudaMemcpyAsync(c->ux_m, ux, N * 8, cudaMemcpyHostToDevice, c->stream));
  else
    LBM_CUDA(c, cudaMemsetAsync(c->ux_m, 0, N * 8, c->stream));
  if (uy)
    LBM_CUDA(c, cudaMemcpyAsync(c->uy_m, uy, N * 8, cudaMemcpyHostToDevice, c->stream));
  else
    LBM_CUDA(c, cudaMemsetAsync(c->uy_m, 0, N * 8, c->stream));
  return init_common(c);
}

lbm_status lbm_init_droplet(lbm_ctx* c, double cx, double cy, double R, double W, double rho_in,
                            double rho_out) {
  if (!c) return LBM_EINVAL;
  if (c->status) return c->status;
  if (!(W > 0) || !(rho_in > 0) || !(rho_out > 0) || !is_fin(cx) || !is_fin(cy) || !is_fin(R))
    return LBM_EINVAL;
  if (c->rho_ref_auto) {
    c->p.rho_ref = rho_in < rho_out ? rho_in : rho_out;
    finalize_consts(c->p);
  }
  LBM_CUDA(c, launch_droplet_rho(c->p, cx, cy, R, W, rho_in, rho_out, c->rho_m, c->ux_m, c->uy_m,
                                 c->stream));
  return init_common(c);
}

lbm_status lbm_step(lbm_ctx* c, int32_t n) {
  if (!c) return LBM_EINVAL;
  if (c->status) return c->status;
  if (n < 0) return LBM_EINVAL;
  if (!c->initialized) return fail(c, LBM_ESTATE, "lbm_step before initialisation");
  while (n >= c->graph_steps) {
    if (!c->graph[c->cur]) {
      lbm_status st = build_graph(c, c->cur);
      if (st != LBM_OK) return st;
    }
    LBM_CUDA(c, cudaGraphLaunch(c->graph[c->cur], c->stream));
    n -= c->graph_steps;
    c->steps += c->graph_steps;  // even: parity unchanged
  }
  for (; n > 0; --n) {
    lbm_status st = launch_one_step(c, c->stream, c->cur);
    if (st != LBM_OK) return st;
    c->cur = 1 - c->cur;
    ++c->steps;
  }
  return LBM_OK;
}

lbm_status lbm_step_timed(lbm_ctx* c, int32_t n, double* ms_step, double* ms_bnd,
                          double* ms_total) {
  if (!c) return LBM_EINVAL;
  if (c->status) return c->status;
  if (n < 1) return LBM_EINVAL;
  if (!c->initialized) return fail(c, LBM_ESTATE, "lbm_step_timed before initialisation");
  std::vector<cudaEvent_t> ev(2 * (size_t)n + 1);
  for (auto& e : ev) LBM_CUDA(c, cudaEventCreate(&e));
  lbm_status st = LBM_OK;
  LBM_CUDA(c, cudaEventRecord(ev[0], c->stream));
  for (int k = 0; k < n && st == LBM_OK; ++k) {
    const int cur = c->cur;
    cudaError_t e = launch_bulk(c, c->stream, cur);
    if (e != cudaSuccess) st = cuda_fail(c, e, "step kernel launch");
    if (st == LBM_OK) cudaEventRecord(ev[2 * k + 1], c->stream);
    if (st == LBM_OK) {
      e = launch_boundary(c->precision, c->p, (int)c->nb, c->bnode, c->boff, c->ldir, c->recipe,
                          c->f[cur], c->f[1 - cur], c->rho_m, c->ux_m, c->uy_m, c->carry,
                          c->track_force ? c->force : nullptr, c->stream);
      if (e != cudaSuccess) st = cuda_fail(c, e, "boundary kernel launch");
    }
    if (st == LBM_OK && c->open_x) {
      e = launch_open_x(c->precision, c->p, c->f[1 - cur], c->flags, c->u_in, c->stream);
      if (e != cudaSuccess) st = cuda_fail(c, e, "channel-end kernel launch");
    }
    if (st == LBM_OK) cudaEventRecord(ev[2 * k + 2], c->stream);
    c->cur = 1 - cur;
    ++c->steps;
  }
  if (st == LBM_OK) {
    cudaError_t e = cudaEventSynchronize(ev[2 * n]);
    if (e != cudaSuccess) st = cuda_fail(c, e, "cudaEventSynchronize");
  }
  if (st == LBM_OK) {
    double s1 = 0, s2 = 0;
    for (int k = 0; k < n; ++k) {
      float a = 0, b = 0;
      cudaEventElapsedTime(&a, ev[2 * k], ev[2 * k + 1]);
      cudaEventElapsedTime(&b, ev[2 * k + 1], ev[2 * k + 2]);
      s1 += a;
      s2 += b;
    }
    float tot = 0;
    cudaEventElapsedTime(&tot, ev[0], ev[2 * n]);
    if (ms_step) *ms_step = s1;
    if (ms_bnd) *ms_bnd = s2;
    if (ms_total) *ms_total = tot;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return st;
}

lbm_status lbm_mass(lbm_ctx* c, double* out) {
  if (!c || !out) return LBM_EINVAL;
  if (c->status) return c->status;
  if (!c->initialized) return fail(c, LBM_ESTATE, "lbm_mass before initialisation");
  LBM_CUDA(c, launch_mass(c->precision, c->p, c->f[c->cur], c->flags, c->partials,
                          c->ledger_blocks, c->mass_out, c->err_flag, c->stream));
  double m = 0;
  int err = 0;
  LBM_CUDA(c, cudaMemcpyAsync(&m, c->mass_out, 8, cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaMemcpyAsync(&err, c->err_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  *out = m;
  if (err & kErrTimeout) return fail(c, LBM_ETIMEOUT, "a bounded wait for a tile copy expired");
  if (err) return fail(c, LBM_EUNSTABLE, "non-positive or non-finite density in the fluid");
  return LBM_OK;
}

lbm_status lbm_fields_device(lbm_ctx* c, double* rho, double* ux, double* uy) {
  if (!c || !rho || !ux || !uy) return LBM_EINVAL;
  if (c->status) return c->status;
  if (!c->initialized) return fail(c, LBM_ESTATE, "lbm_fields before initialisation");
  LBM_CUDA(c, launch_step(c->precision, c->p, c->f[c->cur], nullptr, c->flags, rho, ux, uy, true,
                          c->stream, c->kernel_path));
  return LBM_OK;
}

lbm_status lbm_fields(lbm_ctx* c, double* rho, double* ux, double* uy) {
  if (!c || !rho || !ux || !uy) return LBM_EINVAL;
  if (c->status) return c->status;
  lbm_status st = lbm_fields_device(c, c->rho_m, c->ux_m, c->uy_m);
  if (st != LBM_OK) return st;
  const size_t N = (size_t)c->p.N;
  LBM_CUDA(c, cudaMemcpyAsync(rho, c->rho_m, N * 8, cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaMemcpyAsync(ux, c->ux_m, N * 8, cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaMemcpyAsync(uy, c->uy_m, N * 8, cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_flags(lbm_ctx* c, uint8_t* flags) {
  if (!c || !flags) return LBM_EINVAL;
  if (c->status) return c->status;
  const size_t N = (size_t)c->p.N;
  LBM_CUDA(c, cudaMemcpyAsync(flags, c->flags, N, cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  for (size_t k = 0; k < N; ++k) flags[k] &= (FLAG_SOLID | FLAG_BOUNDARY);
  return LBM_OK;
}

lbm_status lbm_links(lbm_ctx* c, int32_t* node, uint8_t* dir, double* q, int64_t* n_inout) {
  if (!c || !n_inout) return LBM_EINVAL;
  if (c->status) return c->status;
  const int64_t cap = *n_inout;
  *n_inout = c->nl;
  if (!node && !dir && !q) return LBM_OK;
  if (cap < c->nl) return LBM_EINVAL;
  if (c->nl == 0) return LBM_OK;
  std::vector<int32_t> bn(c->nb), bo(c->nb + 1);
  std::vector<uint8_t> ld(c->nl);
  std::vector<double> qq(c->nl);
  LBM_CUDA(c, cudaMemcpyAsync(bn.data(), c->bnode, c->nb * 4, cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaMemcpyAsync(bo.data(), c->boff, (c->nb + 1) * 4, cudaMemcpyDeviceToHost,
                              c->stream));
  LBM_CUDA(c, cudaMemcpyAsync(ld.data(), c->ldir, c->nl, cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaMemcpyAsync(qq.data(), c->lq, c->nl * 8, cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  for (long long b = 0; b < c->nb; ++b)
    for (int l = bo[b]; l < bo[b + 1]; ++l) {
      if (node) node[l] = bn[b];
      if (dir) dir[l] = ld[l];
      if (q) q[l] = qq[l];
    }
  return LBM_OK;
}

lbm_status lbm_info(lbm_ctx* c, lbm_info_t* o) {
  if (!c || !o) return LBM_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->nx = c->p.nx;
  o->ny = c->p.ny;
  o->n_fluid = c->n_fluid;
  o->n_boundary_nodes = c->nb;
  o->n_links = c->nl;
  o->steps = c->steps;
  o->device_bytes = (int64_t)c->device_bytes;
  o->fallbacks = 0;
  o->T = c->T;
  o->psi_wall = c->p.psi_wall;
  return LBM_OK;
}

lbm_status lbm_set_inflow(lbm_ctx* c, double u_in) {
  if (!c) return LBM_EINVAL;
  if (c->status) return c->status;
  if (!std::isfinite(u_in) || std::fabs(u_in) >= 0.5)
    return fail(c, LBM_EINVAL, "inflow velocity must be finite and below 0.5 in lattice units");
  if (c->p.eos != LBM_EOS_NONE)
    return fail(c, LBM_EINVAL, "channel ends are for single-phase flows (eos kind NONE)");
  if (c->p.nx < 3) return fail(c, LBM_EINVAL, "a channel needs nx >= 3");
  for (int k = 0; k < 2; ++k)  // the captured steps do not contain the channel-end pass
    if (c->graph[k]) {
      cudaGraphExecDestroy(c->graph[k]);
      c->graph[k] = nullptr;
    }
  c->open_x = true;
  c->u_in = u_in;
  c->track_force = true;
  return LBM_OK;
}

lbm_status lbm_force(lbm_ctx* c, double* fx, double* fy) {
  if (!c || !fx || !fy) return LBM_EINVAL;
  if (c->status) return c->status;
  if (!c->track_force)
    return fail(c, LBM_ESTATE, "the force is not recorded (lbm_options.track_force)");
  double sx = 0.0, sy = 0.0;
  if (c->nb > 0) {
    std::vector<double> h(2 * c->nb);
    LBM_CUDA(c, cudaMemcpyAsync(h.data(), c->force, c->nb * 16, cudaMemcpyDeviceToHost,
                                c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    for (long long b = 0; b < c->nb; ++b) {  // boundary nodes in ascending order
      sx += h[2 * b];
      sy += h[2 * b + 1];
    }
  }
  *fx = sx;
  *fy = sy;
  return LBM_OK;
}

lbm_status lbm_selftest_bounded_wait(int64_t limit_ns, int32_t complete, void* stream,
                                     int32_t* completed) {
  if (!completed || limit_ns <= 0 || limit_ns > 10000000000LL) return LBM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int* d = nullptr;
  if (cudaMallocAsync(&d, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ENOMEM;
  }
  int h = -1;
  cudaError_t e = launch_wait_selftest((unsigned long long)limit_ns, complete ? 1 : 0, d, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(d, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LBM_ECUDA;
  }
  *completed = h;
  return h == 1 ? LBM_OK : LBM_ETIMEOUT;
}

namespace {

// Header of a state blob (lbm_save_state); the populations and the carry follow it.
struct StateHeader {
  char magic[8];  // "LBMSTAT1"
  int32_t nx, ny, precision, scheme, eos_kind, open_x;
  double tau, rho_ref, u_in;
  int64_t steps, lattice_bytes, nb;
};
constexpr char kStateMagic[8] = {'L', 'B', 'M', 'S', 'T', 'A', 'T', '1'};

int64_t state_bytes(const lbm_ctx* c) {
  return (int64_t)sizeof(StateHeader) + (int64_t)c->lattice_bytes + 8 * (int64_t)c->nb;
}

}  // namespace

lbm_status lbm_state_bytes(const lbm_ctx* c, int64_t* bytes) {
  if (!c || !bytes) return LBM_EINVAL;
  *bytes = state_bytes(c);
  return LBM_OK;
}

lbm_status lbm_save_state(lbm_ctx* c, void* buf, int64_t bytes) {
  if (!c || !buf) return LBM_EINVAL;
  if (c->status) return c->status;
  if (!c->initialized) return fail(c, LBM_ESTATE, "lbm_save_state before any initialisation");
  if (bytes < state_bytes(c)) return fail(c, LBM_EINVAL, "state buffer too small");
  StateHeader h{};
  std::memcpy(h.magic, kStateMagic, 8);
  h.nx = c->p.nx;
  h.ny = c->p.ny;
  h.precision = c->precision;
  h.scheme = c->p.scheme;
  h.eos_kind = c->p.eos;
  h.open_x = c->open_x ? 1 : 0;
  h.tau = c->p.tau;
  h.rho_ref = c->p.rho_ref;
  h.u_in = c->u_in;
  h.steps = c->steps;
  h.lattice_bytes = (int64_t)c->lattice_bytes;
  h.nb = c->nb;
  unsigned char* out = static_cast<unsigned char*>(buf);
  std::memcpy(out, &h, sizeof(h));
  LBM_CUDA(c, cudaMemcpyAsync(out + sizeof(h), c->f[c->cur], c->lattice_bytes,
                              cudaMemcpyDeviceToHost, c->stream));
  if (c->nb > 0)
    LBM_CUDA(c, cudaMemcpyAsync(out + sizeof(h) + c->lattice_bytes, c->carry, 8 * c->nb,
                                cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_load_state(lbm_ctx* c, const void* buf, int64_t bytes) {
  if (!c || !buf) return LBM_EINVAL;
  if (c->status) return c->status;
  if (c->in_batch)
    return fail(c, LBM_ESTATE, "lbm_load_state on a lattice that belongs to a batch");
  if (bytes < (int64_t)sizeof(StateHeader)) return fail(c, LBM_EINVAL, "state blob too short");
  StateHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, kStateMagic, 8) != 0 || h.nx != c->p.nx || h.ny != c->p.ny ||
      h.precision != c->precision || h.scheme != c->p.scheme || h.eos_kind != c->p.eos ||
      std::memcmp(&h.tau, &c->p.tau, sizeof(double)) != 0 ||
      h.lattice_bytes != (int64_t)c->lattice_bytes || h.nb != c->nb || h.steps < 0 ||
      bytes < state_bytes(c))
    return fail(c, LBM_EINVAL, "not a state blob of this lattice");
  if (h.open_x && (!std::isfinite(h.u_in) || std::fabs(h.u_in) >= 0.5))
    return fail(c, LBM_EINVAL, "state blob with an invalid inflow velocity");
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  LBM_CUDA(c, cudaMemcpyAsync(c->f[0], in + sizeof(h), c->lattice_bytes, cudaMemcpyHostToDevice,
                              c->stream));
  LBM_CUDA(c, cudaMemsetAsync(c->f[1], 0, c->lattice_bytes, c->stream));
  if (c->nb > 0)
    LBM_CUDA(c, cudaMemcpyAsync(c->carry, in + sizeof(h) + c->lattice_bytes, 8 * c->nb,
                                cudaMemcpyHostToDevice, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  const bool open_changed = (h.open_x != 0) != c->open_x;
  c->p.rho_ref = h.rho_ref;
  finalize_consts(c->p);
  // captured steps hold the kernel parameters by value and the channel pass or not
  if (c->p.rho_ref != c->graph_rho_ref || open_changed)
    for (int k = 0; k < 2; ++k)
      if (c->graph[k]) {
        cudaGraphExecDestroy(c->graph[k]);
        c->graph[k] = nullptr;
      }
  c->open_x = h.open_x != 0;
  c->u_in = h.u_in;
  if (c->open_x) c->track_force = true;
  c->cur = 0;
  c->steps = h.steps;
  c->initialized = true;
  return LBM_OK;
}

}  // extern "C"
