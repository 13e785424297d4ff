// Batches of lattices advanced together (C ABI lbm_batch_*, declared in include/lbm_gb300.h).
//
// Every lattice of a batch is an ordinary context (its own geometry, link list, two lattices),
// created by lbm_create with the batch's precision, stream and allocation hook.  One time step of
// the batch is three launches whatever the number of lattices:
//   batch_step_kernel      persistent grid over a queue of tiles (lattice, x0, y0)
//   batch_boundary_kernel  persistent grid of 8-lane groups over (lattice, boundary node) items
//   batch_advance_kernel   flips each lattice's current buffer and counts down its step budget
// The tables live at fixed device addresses and the number of tiles and items is read on the
// device, so a captured CUDA graph stays valid while lattices join and leave; lattices whose
// budget is spent are skipped.  The tuner picks the tile height and the queue's schedule (how
// CTAs take tiles, in which order the lattices' tiles stand).  The per-node arithmetic is the single-lattice arithmetic, so a
// lattice gives the same bits alone and inside any batch, with any tile shape.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "lbm_internal.h"

using namespace lbm;

struct lbm_batch {
  int precision = LBM_FP64;
  int eos = LBM_EOS_NONE;
  int max_domains = 0;
  lbm_options opt{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  std::vector<lbm_ctx*> slots;
  std::vector<BatchDomain> h_doms;
  std::vector<char> uploaded;  // slot's entry in the device table is current
  // device tables
  BatchDomain* d_doms = nullptr;
  int* d_counts = nullptr;  // [0] tiles, [1] boundary items, [2] tile claim counter
  int4* d_tiles = nullptr;
  int2* d_items = nullptr;
  int cap_tiles = 0, cap_items = 0;
  std::vector<std::pair<void*, size_t>> blocks;
  int n_tiles = 0, n_items = 0;
  int ry = 0;  // tile rows per thread (tile height 8 ry)
  int sched = LBM_SCHED_STRIDED;  // lbm_schedule of the tile queue
  std::vector<lbm_tune_trial> trials;  // of the last lbm_batch_tune
  int step_grid = 0, bnd_grid = 0;
  bool dirty = true;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 16;
  lbm_status status = LBM_OK;
  std::string msg;
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status s, const std::string& m) {
  if (b && b->status == LBM_OK) {
    b->status = s;
    b->msg = m;
  }
  return s;
}

#define BCUDA(b, call)                                                          \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess)                                                      \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, \
                   std::string(#call) + ": " + cudaGetErrorString(e_));         \
  } while (0)

void* balloc(lbm_batch* b, size_t bytes) {
  void* p = nullptr;
  if (b->opt.alloc) {
    p = b->opt.alloc(bytes, b->opt.alloc_user);
  } else if (cudaMallocAsync(&p, bytes, b->stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) b->blocks.emplace_back(p, bytes);
  return p;
}

void bfree(lbm_batch* b, void* p) {
  for (size_t k = 0; k < b->blocks.size(); ++k)
    if (b->blocks[k].first == p) {
      cudaStreamSynchronize(b->stream);
      if (b->opt.free)
        b->opt.free(p, b->opt.alloc_user);
      else
        cudaFreeAsync(p, b->stream);
      b->blocks.erase(b->blocks.begin() + k);
      return;
    }
}

void drop_graph(lbm_batch* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

// Bring cur / steps_left / steps_done of every lattice from the device into h_doms.
lbm_status sync_down(lbm_batch* b) {
  if (!b->d_doms) return LBM_OK;
  std::vector<BatchDomain> tmp(b->max_domains);
  BCUDA(b, cudaMemcpyAsync(tmp.data(), b->d_doms, sizeof(BatchDomain) * b->max_domains,
                           cudaMemcpyDeviceToHost, b->stream));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  for (int d = 0; d < b->max_domains; ++d) {
    if (!b->slots[d] || !b->uploaded[d]) continue;
    b->h_doms[d].cur = tmp[d].cur;
    b->h_doms[d].steps_left = tmp[d].steps_left;
    b->h_doms[d].steps_done = tmp[d].steps_done;
    b->slots[d]->cur = tmp[d].cur;
    b->slots[d]->steps = tmp[d].steps_done;
  }
  return LBM_OK;
}

BatchDomain describe(lbm_ctx* c, long long steps) {
  BatchDomain d{};
  d.p = c->p;
  d.f[0] = c->f[0];
  d.f[1] = c->f[1];
  d.flags = c->flags;
  d.rho_m = c->rho_m;
  d.ux_m = c->ux_m;
  d.uy_m = c->uy_m;
  d.bnode = c->bnode;
  d.boff = c->boff;
  d.ldir = c->ldir;
  d.recipe = c->recipe;
  d.carry = c->carry;
  d.nb = (int)c->nb;
  d.cur = c->cur;
  d.steps_left = steps;
  d.steps_done = c->steps;
  return d;
}

int* claim_counter(lbm_batch* b) {
  return b->sched == LBM_SCHED_STRIDED ? nullptr : b->d_counts + 2;
}

// Rebuild the tile and item tables from the active lattices and upload everything.  The tiles
// of a lattice stand together in row-major order; the lattices follow in slot order, or by tile
// count, largest first, for LBM_SCHED_CLAIM_LARGEST_FIRST (ties in slot order).
lbm_status upload_tables(lbm_batch* b) {
  const int TH = batch_tile_rows(b->ry), TW = batch_tile_cols();
  std::vector<int> order;
  for (int d = 0; d < b->max_domains; ++d)
    if (b->slots[d]) order.push_back(d);
  auto n_tiles_of = [&](int d) {
    const lbm_ctx* c = b->slots[d];
    return (long long)((c->p.nx + TW - 1) / TW) * ((c->p.ny + TH - 1) / TH);
  };
  if (b->sched == LBM_SCHED_CLAIM_LARGEST_FIRST)
    std::stable_sort(order.begin(), order.end(),
                     [&](int u, int v) { return n_tiles_of(u) > n_tiles_of(v); });
  std::vector<int4> tiles;
  std::vector<int2> items;
  for (int d : order) {
    lbm_ctx* c = b->slots[d];
    for (int y0 = 0; y0 < c->p.ny; y0 += TH)
      for (int x0 = 0; x0 < c->p.nx; x0 += TW) tiles.push_back(make_int4(d, x0, y0, 0));
    for (int k = 0; k < (int)c->nb; ++k) items.push_back(make_int2(d, k));
  }
  if ((int)tiles.size() > b->cap_tiles) {
    drop_graph(b);
    if (b->d_tiles) bfree(b, b->d_tiles);
    b->cap_tiles = (int)tiles.size() * 2 + 1024;
    b->d_tiles = (int4*)balloc(b, sizeof(int4) * b->cap_tiles);
    if (!b->d_tiles) return bfail(b, LBM_ENOMEM, "tile table");
  }
  if ((int)items.size() > b->cap_items) {
    drop_graph(b);
    if (b->d_items) bfree(b, b->d_items);
    b->cap_items = (int)items.size() * 2 + 1024;
    b->d_items = (int2*)balloc(b, sizeof(int2) * b->cap_items);
    if (!b->d_items) return bfail(b, LBM_ENOMEM, "item table");
  }
  b->n_tiles = (int)tiles.size();
  b->n_items = (int)items.size();
  int counts[3] = {b->n_tiles, b->n_items, 0};
  if (!tiles.empty())
    BCUDA(b, cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(int4) * tiles.size(),
                             cudaMemcpyHostToDevice, b->stream));
  if (!items.empty())
    BCUDA(b, cudaMemcpyAsync(b->d_items, items.data(), sizeof(int2) * items.size(),
                             cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaMemcpyAsync(b->d_counts, counts, sizeof(counts), cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaMemcpyAsync(b->d_doms, b->h_doms.data(), sizeof(BatchDomain) * b->max_domains,
                           cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  for (int d = 0; d < b->max_domains; ++d) b->uploaded[d] = b->slots[d] != nullptr;
  b->dirty = false;
  return LBM_OK;
}

lbm_status one_step(lbm_batch* b, cudaStream_t s, cudaEvent_t e_mid = nullptr,
                    cudaEvent_t e_end = nullptr) {
  BCUDA(b, launch_batch_step(b->precision, b->eos, b->ry, b->d_doms, b->d_tiles, b->d_counts,
                             claim_counter(b), b->step_grid, s));
  if (e_mid) BCUDA(b, cudaEventRecord(e_mid, s));
  BCUDA(b, launch_batch_boundary(b->precision, b->d_doms, b->d_items, b->d_counts + 1,
                                 b->bnd_grid, s));
  BCUDA(b, launch_batch_advance(b->d_doms, b->max_domains, b->d_counts + 2, s));
  if (e_end) BCUDA(b, cudaEventRecord(e_end, s));
  return LBM_OK;
}

lbm_status ready(lbm_batch* b) {
  if (b->status) return b->status;
  if (b->dirty) return upload_tables(b);
  return LBM_OK;
}

bool valid_slot(lbm_batch* b, int slot) {
  return b && slot >= 0 && slot < b->max_domains && b->slots[slot];
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(int32_t precision, int32_t eos_kind, int32_t max_domains,
                            const lbm_options* opt, lbm_batch** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (precision < LBM_FP64 || precision > LBM_FP16_DEV) return LBM_EINVAL;
  if (eos_kind < LBM_EOS_NONE || eos_kind > LBM_EOS_CS) return LBM_EINVAL;
  if (max_domains < 1 || max_domains > (1 << 20)) return LBM_EINVAL;
  if (opt && ((opt->alloc == nullptr) != (opt->free == nullptr))) return LBM_EINVAL;
  lbm_batch* b = new lbm_batch();
  b->precision = precision;
  b->eos = eos_kind;
  b->max_domains = max_domains;
  if (opt) b->opt = *opt;
  b->opt.precision = precision;
  b->opt.graph_steps = 0;
  b->stream = (cudaStream_t)b->opt.stream;
  b->slots.assign(max_domains, nullptr);
  b->h_doms.assign(max_domains, BatchDomain{});
  b->uploaded.assign(max_domains, 0);
  // 32-row tiles (FP64: 16), claimed: the fastest pair on the 512-lattice workload
  b->ry = precision == LBM_FP64 ? 2 : 4;
  b->sched = LBM_SCHED_CLAIM;
  b->step_grid = batch_step_grid(precision, eos_kind, b->ry);
  b->bnd_grid = batch_boundary_grid(precision);
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return LBM_ECUDA;
  }
  b->d_doms = (BatchDomain*)balloc(b, sizeof(BatchDomain) * max_domains);
  b->d_counts = (int*)balloc(b, 256);
  if (!b->d_doms || !b->d_counts) {
    lbm_batch_destroy(b);
    return LBM_ENOMEM;
  }
  if (cudaMemsetAsync(b->d_doms, 0, sizeof(BatchDomain) * max_domains, b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_counts, 0, 256, b->stream) != cudaSuccess) {
    cudaGetLastError();
    lbm_batch_destroy(b);
    return LBM_ECUDA;
  }
  *out = b;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (auto& c : b->slots)
    if (c) lbm_destroy(c);
  b->slots.clear();
  while (!b->blocks.empty()) bfree(b, b->blocks.back().first);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->msg.c_str() : "null batch"; }

lbm_status lbm_batch_add(lbm_batch* b, const lbm_domain* d, int64_t steps, int32_t* slot) {
  if (!b || !d || !slot || steps < 0) return LBM_EINVAL;
  if (b->status) return b->status;
  if (d->eos.kind != b->eos) return LBM_EINVAL;
  int free_slot = -1;
  for (int k = 0; k < b->max_domains; ++k)
    if (!b->slots[k]) {
      free_slot = k;
      break;
    }
  if (free_slot < 0) return LBM_ENOMEM;
  lbm_ctx* c = nullptr;
  lbm_status st = lbm_create(&d->geometry, &d->eos, d->tau, d->scheme, &b->opt, &c);
  if (st != LBM_OK) return st;
  c->in_batch = true;
  if (d->init == 1)
    st = lbm_init_droplet(c, d->cx, d->cy, d->R, d->W, d->rho_in, d->rho_out);
  else {
    std::vector<double> rho((size_t)c->p.N, d->rho_in);
    st = lbm_init_fields(c, rho.data(), nullptr, nullptr);
  }
  if (st != LBM_OK) {
    lbm_destroy(c);
    return st;
  }
  st = sync_down(b);
  if (st != LBM_OK) {
    lbm_destroy(c);
    return st;
  }
  b->slots[free_slot] = c;
  b->h_doms[free_slot] = describe(c, steps);
  b->dirty = true;
  *slot = free_slot;
  return LBM_OK;
}

lbm_status lbm_batch_remove(lbm_batch* b, int32_t slot) {
  if (!valid_slot(b, slot)) return LBM_EINVAL;
  if (b->status) return b->status;
  lbm_status st = sync_down(b);
  if (st != LBM_OK) return st;
  lbm_destroy(b->slots[slot]);
  b->slots[slot] = nullptr;
  b->uploaded[slot] = 0;
  b->h_doms[slot] = BatchDomain{};
  b->dirty = true;
  return LBM_OK;
}

lbm_status lbm_batch_set_steps(lbm_batch* b, int32_t slot, int64_t steps) {
  if (!valid_slot(b, slot) || steps < 0) return LBM_EINVAL;
  if (b->status) return b->status;
  lbm_status st = sync_down(b);
  if (st != LBM_OK) return st;
  b->h_doms[slot].steps_left = steps;
  b->dirty = true;
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int32_t n) {
  if (!b || n < 0) return LBM_EINVAL;
  lbm_status st = ready(b);
  if (st != LBM_OK) return st;
  while (n >= b->graph_steps) {
    if (!b->graph) {
      cudaGraph_t g = nullptr;
      BCUDA(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
      for (int k = 0; k < b->graph_steps && st == LBM_OK; ++k) st = one_step(b, b->cap_stream);
      cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
      if (st != LBM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      BCUDA(b, e);
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      BCUDA(b, e);
    }
    BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
    n -= b->graph_steps;
  }
  for (; n > 0 && st == LBM_OK; --n) st = one_step(b, b->stream);
  return st;
}

lbm_status lbm_batch_step_timed(lbm_batch* b, int32_t n, double* ms_total, double* ms_step_kernel,
                                double* ms_boundary) {
  if (!b || n < 1) return LBM_EINVAL;
  lbm_status st = ready(b);
  if (st != LBM_OK) return st;
  std::vector<cudaEvent_t> ev(2 * (size_t)n + 1);
  for (auto& e : ev) BCUDA(b, cudaEventCreate(&e));
  BCUDA(b, cudaEventRecord(ev[0], b->stream));
  for (int k = 0; k < n && st == LBM_OK; ++k) st = one_step(b, b->stream, ev[2 * k + 1], ev[2 * k + 2]);
  if (st == LBM_OK && cudaEventSynchronize(ev[2 * n]) != cudaSuccess)
    st = bfail(b, LBM_ECUDA, "cudaEventSynchronize");
  if (st == LBM_OK) {
    double s1 = 0, s2 = 0;
    for (int k = 0; k < n; ++k) {
      float x = 0, y = 0;
      cudaEventElapsedTime(&x, ev[2 * k], ev[2 * k + 1]);
      cudaEventElapsedTime(&y, ev[2 * k + 1], ev[2 * k + 2]);
      s1 += x;
      s2 += y;
    }
    float tot = 0;
    cudaEventElapsedTime(&tot, ev[0], ev[2 * n]);
    if (ms_total) *ms_total = tot;
    if (ms_step_kernel) *ms_step_kernel = s1;
    if (ms_boundary) *ms_boundary = s2;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return st;
}

lbm_status lbm_batch_progress(lbm_batch* b, int32_t slot, int64_t* steps_done,
                              int64_t* steps_left) {
  if (!valid_slot(b, slot)) return LBM_EINVAL;
  if (b->status) return b->status;
  lbm_status st = sync_down(b);
  if (st != LBM_OK) return st;
  if (steps_done) *steps_done = b->h_doms[slot].steps_done;
  if (steps_left) *steps_left = b->h_doms[slot].steps_left;
  return LBM_OK;
}

lbm_status lbm_batch_poll(lbm_batch* b, int32_t n, int64_t* steps_left) {
  if (!b || n < 0 || (n > 0 && !steps_left)) return LBM_EINVAL;
  if (b->status) return b->status;
  lbm_status st = sync_down(b);
  if (st != LBM_OK) return st;
  for (int d = 0; d < n; ++d)
    steps_left[d] = (d < b->max_domains && b->slots[d]) ? b->h_doms[d].steps_left : -1;
  return LBM_OK;
}

lbm_status lbm_batch_domain(lbm_batch* b, int32_t slot, lbm_ctx** ctx) {
  if (!valid_slot(b, slot) || !ctx) return LBM_EINVAL;
  if (b->status) return b->status;
  lbm_status st = sync_down(b);
  if (st != LBM_OK) return st;
  *ctx = b->slots[slot];
  return LBM_OK;
}

lbm_status lbm_batch_tune(lbm_batch* b, int32_t trial_steps, int32_t* tile_rows) {
  if (!b || trial_steps < 1) return LBM_EINVAL;
  lbm_status st = ready(b);
  if (st != LBM_OK) return st;
  const int cands[3] = {1, 2, 4};
  const int scheds[3] = {LBM_SCHED_STRIDED, LBM_SCHED_CLAIM, LBM_SCHED_CLAIM_LARGEST_FIRST};
  int best = b->ry, best_sched = b->sched;
  float best_ms = 1e30f;
  b->trials.clear();
  cudaEvent_t e0, e1;
  BCUDA(b, cudaEventCreate(&e0));
  BCUDA(b, cudaEventCreate(&e1));
  // Only the step kernel runs: it writes the not-yet-current buffer of every lattice, which
  // the next real step overwrites, so the state does not change.  The claim counter is zeroed
  // before every launch (the advance kernel does it in a real step), for every schedule alike.
  auto launch = [&](int ry) {
    if (cudaMemsetAsync(b->d_counts + 2, 0, sizeof(int), b->stream) != cudaSuccess ||
        launch_batch_step(b->precision, b->eos, ry, b->d_doms, b->d_tiles, b->d_counts,
                          claim_counter(b), b->step_grid, b->stream) != cudaSuccess)
      st = bfail(b, LBM_ECUDA, "tuning launch");
  };
  for (int ry : cands) {
    if (b->precision == LBM_FP64 && ry == 4) continue;  // register budget of FP64
    for (int sc : scheds) {
      b->ry = ry;
      b->sched = sc;
      b->step_grid = batch_step_grid(b->precision, b->eos, ry);
      st = upload_tables(b);
      if (st != LBM_OK) break;
      for (int k = 0; k < 2 && st == LBM_OK; ++k) launch(ry);  // warm-up
      cudaEventRecord(e0, b->stream);
      for (int k = 0; k < trial_steps && st == LBM_OK; ++k) launch(ry);
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (st != LBM_OK) break;
      b->trials.push_back(lbm_tune_trial{batch_tile_rows(ry), sc, (double)ms / trial_steps});
      if (ms < best_ms) {
        best_ms = ms;
        best = ry;
        best_sched = sc;
      }
    }
    if (st != LBM_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // leave the counter at 0 for the next real step
  if (cudaMemsetAsync(b->d_counts + 2, 0, sizeof(int), b->stream) != cudaSuccess && st == LBM_OK)
    st = bfail(b, LBM_ECUDA, "cudaMemsetAsync");
  if (st != LBM_OK) return st;
  drop_graph(b);
  b->ry = best;
  b->sched = best_sched;
  b->step_grid = batch_step_grid(b->precision, b->eos, best);
  st = upload_tables(b);
  if (tile_rows) *tile_rows = batch_tile_rows(best);
  return st;
}

lbm_status lbm_batch_tune_trials(const lbm_batch* b, int32_t max, lbm_tune_trial* out,
                                 int32_t* n) {
  if (!b || !n || max < 0 || (max > 0 && !out)) return LBM_EINVAL;
  *n = (int32_t)b->trials.size();
  for (int32_t k = 0; k < max && k < *n; ++k) out[k] = b->trials[k];
  return LBM_OK;
}

lbm_status lbm_batch_set_schedule(lbm_batch* b, int32_t tile_rows, int32_t schedule) {
  if (!b) return LBM_EINVAL;
  if (schedule < LBM_SCHED_STRIDED || schedule > LBM_SCHED_CLAIM_LARGEST_FIRST) return LBM_EINVAL;
  int ry = 0;
  for (int r : {1, 2, 4})
    if (batch_tile_rows(r) == tile_rows) ry = r;
  if (ry == 0 || (b->precision == LBM_FP64 && ry == 4)) return LBM_EINVAL;
  if (b->status) return b->status;
  drop_graph(b);
  b->ry = ry;
  b->sched = schedule;
  b->step_grid = batch_step_grid(b->precision, b->eos, ry);
  b->dirty = true;
  return LBM_OK;
}

lbm_status lbm_batch_info(lbm_batch* b, lbm_batch_info_t* o) {
  if (!b || !o) return LBM_EINVAL;
  std::memset(o, 0, sizeof(*o));
  for (auto* c : b->slots) {
    if (!c) continue;
    o->active += 1;
    o->nodes += c->p.N;
    o->fluid_nodes += c->n_fluid;
    o->boundary_links += c->nl;
    o->device_bytes += (int64_t)c->device_bytes;
  }
  for (auto& blk : b->blocks) o->device_bytes += (int64_t)blk.second;
  o->tiles = b->dirty ? -1 : b->n_tiles;
  o->tile_rows = batch_tile_rows(b->ry);
  o->tile_cols = batch_tile_cols();
  o->schedule = b->sched;
  return LBM_OK;
}

lbm_status lbm_domain_bytes(const lbm_domain* d, int32_t precision, int64_t* bytes) {
  if (!d || !bytes || precision < LBM_FP64 || precision > LBM_FP16_DEV) return LBM_EINVAL;
  const int64_t N = (int64_t)d->geometry.nx * d->geometry.ny;
  const int64_t lattice = precision == LBM_FP64 ? 72 * N : (precision == LBM_FP32_DEV ? 36 * N : 20 * N);
  // links: at most 8 per boundary node; a circle of radius r has about 2 pi r + 8 boundary nodes
  double nb = 0;
  for (int k = 0; k < d->geometry.n_circles; ++k) nb += 6.3 * d->geometry.circles[k].r + 8;
  if (d->geometry.wall_q_lo > 0) nb += d->geometry.nx;
  if (d->geometry.wall_q_hi > 0) nb += d->geometry.nx;
  const int64_t links = (int64_t)(8 * nb);
  *bytes = 2 * lattice + N + 24 * N + 12 * 1024 + (int64_t)nb * 24 + links * 70 + 64 * 1024;
  return LBM_OK;
}

}  // extern "C"
