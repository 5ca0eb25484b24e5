// C ABI of the M1 RT subcycle (include/rt.h): context, mesh upload, state
// transfer, the subcycle driver and the stage entry points.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rt.h"
#include "rt_ctx.h"
#include "rt_adjoint.cuh"

using namespace m1rt;

namespace {

constexpr int kThreads = 64;
inline int nblk(long long n, int t = kThreads) { return (int)((n + t - 1) / t); }

thread_local std::string g_create_error;

}  // namespace


namespace {

rt_status fail(rt_ctx* c, rt_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf; else g_create_error = buf;
  return st;
}

rt_status cuda_fail(rt_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(c, RT_OOM, "%s: out of device memory", what);
  }
  return fail(c, RT_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                         \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

template <class T> rt_status dalloc(rt_ctx* ctx, T** p, size_t n, const char* what) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  ctx->allocs.push_back(q);
  *p = (T*)q;
  return RT_OK;
}

void drop_graph(rt_ctx::GraphSlot& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g = rt_ctx::GraphSlot();
}

void free_set(rt_ctx::ActSet& a) {
  for (void* p : a.allocs) cudaFree(p);
  drop_graph(a.graph);
  a = rt_ctx::ActSet();
}

rt_ctx::GraphSlot& cur_graph(rt_ctx* ctx) {
  return ctx->cur_set < 0 ? ctx->all_graph : ctx->sets[ctx->cur_set].graph;
}

// Make set k (-1: every cell active) the current one: the launchers read
// its lists through the context's view fields.
void use_set(rt_ctx* ctx, int k) {
  ctx->cur_set = k;
  if (k < 0) {
    ctx->all_active = true;
    ctx->act_cells = ctx->touched_cells = ctx->act_faces = ctx->grad_blocks = nullptr;
    ctx->touched = nullptr;
    ctx->n_act = ctx->n_touched = ctx->n_act_faces = ctx->n_grad_blocks = 0;
    ctx->grad_cap_list = 0;
    return;
  }
  rt_ctx::ActSet& a = ctx->sets[k];
  a.used = ++ctx->use_clock;
  ctx->all_active = false;
  ctx->act_cells = a.act_cells; ctx->touched_cells = a.touched_cells; ctx->act_faces = a.act_faces;
  ctx->grad_blocks = a.grad_blocks; ctx->touched = a.touched;
  ctx->n_act = a.n_act; ctx->n_touched = a.n_touched; ctx->n_act_faces = a.n_act_faces;
  ctx->n_grad_blocks = a.n_grad_blocks;
  ctx->grad_cap_list = a.grad_cap_list;
}

void free_active(rt_ctx* ctx) {
  for (auto& a : ctx->sets) free_set(a);
  drop_graph(ctx->all_graph);
  use_set(ctx, -1);
}

void free_all(rt_ctx* ctx) {
  ctx->gen++;
  free_active(ctx);
  for (void* p : ctx->allocs) cudaFree(p);
  ctx->allocs.clear();
  ctx->mesh_ready = false;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy n elements from caller memory (host or device) to device memory dst.
rt_status copy_in(rt_ctx* ctx, void* dst, const void* src, size_t bytes) {
  cudaMemcpyKind k = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(dst, src, bytes, k, ctx->stream), "copy in");
  if (k == cudaMemcpyHostToDevice) CK(cudaStreamSynchronize(ctx->stream), "copy in");
  return RT_OK;
}

rt_status copy_out(rt_ctx* ctx, void* dst, const void* src, size_t bytes) {
  cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(dst, src, bytes, k, ctx->stream), "copy out");
  if (k == cudaMemcpyDeviceToHost) CK(cudaStreamSynchronize(ctx->stream), "copy out");
  return RT_OK;
}

bool mixed(const rt_ctx* ctx) { return ctx->cfg.precision == RT_MIXED; }
bool comp_sum(const rt_ctx* ctx) { return ctx->cfg.gather_sum == 1; }

rt_status check_config(const rt_config* c) {
  if (c->n_bins < 1 || c->n_bins > 3) return fail(nullptr, RT_INVALID_ARG, "n_bins must be 1..3");
  if (c->precision != RT_FP64 && c->precision != RT_MIXED) return fail(nullptr, RT_INVALID_ARG, "bad precision");
  if (!(c->c_red > 0) || !(c->unit_length_cm > 0) || !(c->cfl > 0) || c->box < 0)
    return fail(nullptr, RT_INVALID_ARG, "c_red, unit_length_cm and cfl must be > 0, box >= 0");
  if (c->chem_mode < 0 || c->chem_mode > 2) return fail(nullptr, RT_INVALID_ARG, "chem_mode must be 0..2");
  if (c->order < 1 || c->order > 2) return fail(nullptr, RT_INVALID_ARG, "order must be 1 or 2");
  if (c->chem_mode > 0 && (!(c->f_s > 0) || !(c->f_max > 0) || c->max_substeps < 1 || c->x_floor < 0))
    return fail(nullptr, RT_INVALID_ARG, "bad substep parameters");
  if (c->y_he < 0 || c->lim_eps < 0) return fail(nullptr, RT_INVALID_ARG, "y_he and lim_eps must be >= 0");
  if (c->gather_sum < 0 || c->gather_sum > 1) return fail(nullptr, RT_INVALID_ARG, "gather_sum must be 0 or 1");
  if (c->splitting < 0 || c->splitting > 1) return fail(nullptr, RT_INVALID_ARG, "splitting must be 0 or 1");
  if (c->time_order < 1 || c->time_order > 2) return fail(nullptr, RT_INVALID_ARG, "time_order must be 1 or 2");
  return RT_OK;
}

template <class R> Geo<R> geo(const rt_ctx* ctx);
template <> Geo<double> geo<double>(const rt_ctx* c) {
  return Geo<double>{c->C, c->F, c->B, make_divb(c->B), c->off, c->csr, c->nbr, c->lr, c->nA64, c->rL64, c->rR64, c->w64, c->minv64,
                     (const d4*)c->hw, (const d4*)c->hx, (const double*)c->xmax, nullptr, nullptr, c->B,
                     c->touched_cells, c->n_touched,
                     c->grad_blocks, c->n_grad_blocks, c->touched, c->act_faces, c->n_act_faces};
}
template <> Geo<float> geo<float>(const rt_ctx* c) {
  // the FP32 sweep reads faces through fa / fb; no per-array face copies
  return Geo<float>{c->C, c->F, c->B, make_divb(c->B), c->off, c->csr, c->nbr, c->lr, nullptr, nullptr, nullptr, nullptr,
                    c->minv32, (const float4*)c->hw, (const float4*)c->hx, (const float*)c->xmax, c->fa32, c->fb32,
                    pad_bins(c->B),
                    c->touched_cells, c->n_touched, c->grad_blocks, c->n_grad_blocks, c->touched, c->act_faces,
                    c->n_act_faces};
}

ChemParams chem_params(const rt_ctx* ctx) {
  ChemParams P;
  const rt_config& c = ctx->cfg;
  P.B = c.n_bins;
  P.mode = c.chem_mode;
  P.flags = c.chem_flags;
  P.c_red = c.c_red;
  P.y_he = c.y_he;
  P.f_s = c.f_s;
  P.f_max = c.f_max;
  P.x_floor = c.x_floor;
  P.max_sub = c.max_substeps;
  P.smask = P.emask = 0;
  for (int b = 0; b < kMaxBins; ++b)
    for (int s = 0; s < 3; ++s) {
      P.sigma[b][s] = b < c.n_bins ? c.sigma[b][s] : 0.0;
      P.eps[b][s] = b < c.n_bins ? c.eps[b][s] : 0.0;
      if (P.sigma[b][s] != 0.0) P.smask |= 1 << (3 * b + s);
      if (P.eps[b][s] != 0.0) P.emask |= 1 << (3 * b + s);
      P.heat_f[b][s] = (float)(P.eps[b][s] * P.sigma[b][s] / kHeatScale);
    }
  return P;
}

CellArgs cell_args(rt_ctx* ctx, double dt, int gather, int inject, int chem) {
  CellArgs a;
  a.C = ctx->C; a.B = ctx->B; a.divB = make_divb(ctx->B); a.off = ctx->off; a.csr = ctx->csr; a.vol = ctx->vol; a.ivol = ctx->ivol; a.rad = ctx->rad;
  a.radN = ctx->radN;
  a.nH = ctx->nH; a.x5 = ctx->x5; a.T = ctx->T; a.src_idx = ctx->src_idx; a.src_rate = ctx->src_rate;
  a.nsub = ctx->nsub; a.status = ctx->status;
  a.lam = ctx->cfg.c_red * dt / ctx->cfg.unit_length_cm;
  a.dt = dt;
  const double lu = ctx->cfg.unit_length_cm;
  a.lu3 = lu * lu * lu;
  a.do_gather = gather;
  a.do_inject = inject && ctx->n_src_cells > 0;
  a.do_chem = chem && ctx->cfg.chem_mode > 0;
  a.rad0 = nullptr;
  a.heun = 0;
  // individual time steps: chemistry over the active cells, the flux
  // application over the cells with an active interface
  a.list = chem ? ctx->act_cells : ctx->touched_cells;
  a.n = chem ? ctx->n_act : ctx->n_touched;
  return a;
}

// ---- kernel launches -------------------------------------------------------

// Start/stop events around one launch of class k when profiling is on.
struct ProfScope {
  rt_ctx* c;
  int k;
  int idx = -1;
  ProfScope(rt_ctx* ctx, int kind) : c(ctx), k(kind) {
    c->launches++;
    if (!c->profiling) return;
    idx = (int)c->ev_used.size() * 2;
    while ((int)c->ev_pool.size() < idx + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) { idx = -1; return; }
      c->ev_pool.push_back(e);
    }
    cudaEventRecord(c->ev_pool[idx], c->stream);
  }
  ~ProfScope() {
    if (idx < 0) return;
    cudaEventRecord(c->ev_pool[idx + 1], c->stream);
    c->ev_used.push_back({k, idx});
  }
};

template <class R> const R4<R>* sweep_rad(rt_ctx* ctx);
template <> const d4* sweep_rad<double>(rt_ctx* ctx) { return ctx->rad; }
template <> const float4* sweep_rad<float>(rt_ctx* ctx) { return ctx->shadow; }

constexpr int kGradNB = 4;   // neighbour loads in flight per thread (staged gradients)
// An active set's gradients run over its touched-cell list when fewer than
// this fraction of the cells of the blocks it touches are touched, else over
// those blocks (measured on the 2e5-cell hierarchy: the list form is faster
// at 32 % and 61 %, slower at 87 %)
constexpr double kGradListDensity = 0.75;
constexpr size_t kGradSmemMax = 160 * 1024;

template <class R> void launch_grad(rt_ctx* ctx) {
  ProfScope ps(ctx, RT_KERNEL_GRAD);
  const R e = (R)ctx->cfg.lim_eps;
  if constexpr (sizeof(R) == 4) {
    if (ctx->grad_cap > 0 && ctx->cfg.order >= 2) {
      // every cell active: blocks of consecutive cells; an active set: blocks
      // of consecutive entries of its touched-cell list (no work for the
      // untouched cells of a block)
      const bool list = !ctx->all_active && ctx->grad_cap_list > 0 &&
                        (double)ctx->n_touched < kGradListDensity * kGradCells * (double)ctx->n_grad_blocks;
      const int cap = list ? ctx->grad_cap_list : ctx->grad_cap;
      const int nb = ctx->all_active ? (ctx->C + kGradCells - 1) / kGradCells
                     : list          ? (ctx->n_touched + kGradCells - 1) / kGradCells
                                     : ctx->n_grad_blocks;
      if (nb == 0) return;
      const size_t smem = 2 * (size_t)cap * sizeof(float4);
      k_grad_staged<kGradNB><<<nb, kGradCells * ctx->B, smem, ctx->stream>>>(
          geo<float>(ctx), sweep_rad<float>(ctx), (float*)ctx->G, ctx->cfg.limiter, e * e, cap, ctx->status,
          list ? 1 : 0);
      return;
    }
  }
  const long long n = (long long)(ctx->all_active ? ctx->C : ctx->n_touched) * ctx->B;
  if (n == 0) return;
  k_grad<R><<<nblk(n), kThreads, 0, ctx->stream>>>(geo<R>(ctx), sweep_rad<R>(ctx), (R*)ctx->G, ctx->cfg.order,
                                                   ctx->cfg.limiter, e * e);
}

template <class R> void launch_flux(rt_ctx* ctx) {
  ProfScope ps(ctx, RT_KERNEL_FLUX);
  const long long n = (long long)(ctx->all_active ? ctx->F : ctx->n_act_faces) * ctx->B;
  if (n == 0) return;
  k_flux<R><<<nblk(n), kThreads, 0, ctx->stream>>>(geo<R>(ctx), sweep_rad<R>(ctx), (const R*)ctx->G,
                                                   (R4<R>*)ctx->flux);
}

template <bool Heun> void launch_gather_k(rt_ctx* ctx, const CellArgs& a, long long n, bool in_l2) {
  const float4* f32 = (const float4*)ctx->flux;
  if (mixed(ctx) && comp_sum(ctx) && in_l2)
    k_gather<float, true, true, Heun><<<nblk(n), kThreads, 0, ctx->stream>>>(a, f32, ctx->shadow);
  else if (mixed(ctx) && comp_sum(ctx))
    k_gather<float, true, false, Heun><<<nblk(n), kThreads, 0, ctx->stream>>>(a, f32, ctx->shadow);
  else if (mixed(ctx))
    k_gather<float, false, false, Heun><<<nblk(n), kThreads, 0, ctx->stream>>>(a, f32, ctx->shadow);
  else
    k_gather<double, false, false, Heun><<<nblk(n), kThreads, 0, ctx->stream>>>(a, (const d4*)ctx->flux, nullptr);
}

// stage: 0 plain update; 1 also keeps the input state in rad0 (first Heun
// stage); 2 forms U/2 + U2/2 with the state kept in rad0 (second stage)
void launch_gather(rt_ctx* ctx, double dt, int stage = 0) {
  ProfScope ps(ctx, RT_KERNEL_GATHER);
  CellArgs a = cell_args(ctx, dt, 1, 0, 0);
  a.rad0 = ctx->rad0;
  a.heun = stage;
  const long long n = (long long)(ctx->all_active ? ctx->C : ctx->n_touched) * ctx->B;
  if (n == 0) return;
  // with the FP32 flux array held in L2 (129 MB on GB300) the predicated form
  const bool in_l2 = (size_t)ctx->F * ctx->B * sizeof(float4) <= ctx->l2_bytes;
  if (stage == 0)
    launch_gather_k<false>(ctx, a, n, in_l2);
  else
    launch_gather_k<true>(ctx, a, n, in_l2);
}

void launch_chem(rt_ctx* ctx, double dt, const ChemTape* tape = nullptr) {
  ProfScope ps(ctx, RT_KERNEL_CHEM);
  CellArgs a = cell_args(ctx, dt, 0, 1, 1);
  ChemParams P = chem_params(ctx);
  const int t = 128;
  const int nc = ctx->all_active ? ctx->C : ctx->n_act;
  if (nc == 0) return;
  if (!mixed(ctx)) {
    // first attempt of every cell, then the rejected cells (as the mixed path)
    k_chem64_first<<<nblk(nc, t), t, 0, ctx->stream>>>(a, P, ctx->work_cell, ctx->work_f1d, ctx->work_ctl);
    if (!a.do_chem) return;
    ctx->launches++;
    const int nb = (int)std::min<long long>(nblk(nc, t), ctx->n_sm);
    if (tape)
      k_chem64_rest<true><<<nb, t, 0, ctx->stream>>>(a, P, ctx->work_cell, ctx->work_f1d, ctx->work_ctl, *tape);
    else
      k_chem64_rest<false><<<nb, t, 0, ctx->stream>>>(a, P, ctx->work_cell, ctx->work_f1d, ctx->work_ctl,
                                                       ChemTape{});
    return;
  }
  // first attempt of every cell, then the rejected cells (a persistent grid
  // of one block per SM that takes the worklist 128 entries at a time; the
  // worklist is short once the gas is near equilibrium)
  ChemWork w{ctx->work_cell, ctx->work_f1, ctx->work_ctl};
  k_chem_first<<<nblk(nc, t), t, 0, ctx->stream>>>(a, P, ctx->shadow, w);
  if (!a.do_chem) return;
  ctx->launches++;
  const int nb = (int)std::min<long long>(nblk(nc, t), ctx->n_sm);
  k_chem_rest<<<nb, t, 0, ctx->stream>>>(a, P, ctx->shadow, w);
}

void launch_grad_any(rt_ctx* ctx) { mixed(ctx) ? launch_grad<float>(ctx) : launch_grad<double>(ctx); }
void launch_flux_any(rt_ctx* ctx) { mixed(ctx) ? launch_flux<float>(ctx) : launch_flux<double>(ctx); }

// Transport over dt with the configured integrator: one forward-Euler
// stage, or Heun's two stages with the combination fused into the second
// flux application.
void transport(rt_ctx* ctx, double dt) {
  const bool heun = ctx->cfg.time_order == 2;
  launch_grad_any(ctx);
  launch_flux_any(ctx);
  launch_gather(ctx, dt, heun ? 1 : 0);
  if (!heun) return;
  launch_grad_any(ctx);
  launch_flux_any(ctx);
  launch_gather(ctx, dt, 2);
}

// Mixed precision: the state (radN, FP32 sweep records) from the interface
// records in ctx->rad, and back.
void refresh_shadow(rt_ctx* ctx) {
  if (!mixed(ctx)) return;
  long long n = (long long)ctx->C * ctx->B;
  k_split_rad<<<nblk(n), kThreads, 0, ctx->stream>>>((int)n, ctx->rad, ctx->radN, ctx->shadow);
}
void join_state(rt_ctx* ctx) {
  if (!mixed(ctx)) return;
  long long n = (long long)ctx->C * ctx->B;
  k_join_rad<<<nblk(n), kThreads, 0, ctx->stream>>>((int)n, ctx->radN, ctx->shadow, ctx->rad);
}

rt_status launched(rt_ctx* ctx, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  return RT_OK;
}

rt_status need_mesh(rt_ctx* ctx) {
  if (!ctx) return fail(nullptr, RT_INVALID_ARG, "null context");
  if (!ctx->mesh_ready) return fail(ctx, RT_NOT_READY, "rt_init_mesh has not succeeded");
  return RT_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

rt_status rt_create(const rt_config* cfg, void* stream, rt_ctx** out) {
  if (!out) return fail(nullptr, RT_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(nullptr, RT_INVALID_ARG, "cfg is NULL");
  rt_status st = check_config(cfg);
  if (st) return st;
  rt_ctx* ctx = new rt_ctx;
  ctx->cfg = *cfg;
  ctx->stream = (cudaStream_t)stream;
  ctx->B = cfg->n_bins;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e != cudaSuccess) {
    delete ctx;
    cudaGetLastError();
    return fail(nullptr, RT_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  }
  if (cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess ||
      ctx->n_sm < 1) {
    cudaGetLastError();
    ctx->n_sm = 1;
  }
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device) != cudaSuccess || l2 < 0) {
    cudaGetLastError();
    l2 = 0;
  }
  ctx->l2_bytes = (size_t)l2;
  *out = ctx;
  return RT_OK;
}

rt_status rt_set_stream(rt_ctx* ctx, void* stream) {
  if (!ctx) return fail(nullptr, RT_INVALID_ARG, "null context");
  ctx->stream = (cudaStream_t)stream;
  ctx->gen++;
  return RT_OK;
}

rt_status rt_init_mesh(rt_ctx* ctx, const rt_cells* cells, const rt_faces* faces) {
  if (!ctx) return fail(nullptr, RT_INVALID_ARG, "null context");
  if (!cells || !faces) return fail(ctx, RT_INVALID_ARG, "cells or faces is NULL");
  if (cells->n <= 0 || faces->n < 0 || cells->n > (1LL << 30) || faces->n > (1LL << 29))
    return fail(ctx, RT_INVALID_ARG, "cell or face count out of range");
  if (!cells->volume || !cells->cx || !cells->cy || !cells->cz || !faces->left || !faces->right || !faces->area ||
      !faces->nx || !faces->ny || !faces->nz || !faces->fx || !faces->fy || !faces->fz)
    return fail(ctx, RT_INVALID_ARG, "mesh array is NULL");
  free_all(ctx);
  const int C = (int)cells->n, F = (int)faces->n, B = ctx->B;
  ctx->C = C;
  ctx->F = F;
  // host copies for validation and the CSR build (these are the only host
  // passes over the mesh)
  std::vector<int32_t> L(F), Rr(F);
  std::vector<double> V(C);
  const bool dev_l = F > 0 && is_device_ptr(faces->left);
  if (F > 0) {
    CK(cudaMemcpy(L.data(), faces->left, F * 4, dev_l ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost), "mesh");
    CK(cudaMemcpy(Rr.data(), faces->right, F * 4,
                  is_device_ptr(faces->right) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost), "mesh");
  }
  CK(cudaMemcpy(V.data(), cells->volume, (size_t)C * 8,
                is_device_ptr(cells->volume) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost), "mesh");
  std::vector<int32_t> off(C + 1, 0);
  for (int f = 0; f < F; ++f) {
    if (L[f] < 0 || L[f] >= C || Rr[f] < 0 || Rr[f] >= C || L[f] == Rr[f])
      return fail(ctx, RT_BAD_MESH, "face %d joins cells %d and %d (C = %d)", f, L[f], Rr[f], C);
    off[L[f] + 1]++;
    off[Rr[f] + 1]++;
  }
  double minV = INFINITY;
  for (int i = 0; i < C; ++i) {
    if (!(V[i] > 0) || !std::isfinite(V[i])) return fail(ctx, RT_BAD_MESH, "cell %d has volume %g", i, V[i]);
    minV = std::min(minV, V[i]);
  }
  int maxdeg = 0;
  for (int i = 0; i < C; ++i) {
    maxdeg = std::max(maxdeg, off[i + 1]);
    off[i + 1] += off[i];
  }
  for (int i = 0; i < C; ++i) {
    if (off[i + 1] == off[i]) return fail(ctx, RT_BAD_MESH, "cell %d has no faces", i);
  }
  std::vector<int32_t> csr(2 * (size_t)F), nbr(2 * (size_t)F);
  {
    std::vector<int32_t> fill(off.begin(), off.end() - 1);
    for (int f = 0; f < F; ++f) {     // ascending face index within each cell
      nbr[fill[L[f]]] = Rr[f];
      csr[fill[L[f]]++] = f << 1;
      nbr[fill[Rr[f]]] = L[f];
      csr[fill[Rr[f]]++] = (f << 1) | 1;
    }
  }
  ctx->max_deg = maxdeg;
  ctx->min_dx_cm = std::cbrt(minV) * ctx->cfg.unit_length_cm;
  // staged gradients (FP32 sweep): shared memory for the largest block's
  // half-edge records; a mesh whose blocks need more than kGradSmemMax keeps
  // the unstaged kernel
  ctx->grad_cap = 0;
  if (mixed(ctx)) {
    int cap = 0;
    for (int c0 = 0; c0 < C; c0 += kGradCells) cap = std::max(cap, off[std::min(c0 + kGradCells, C)] - off[c0]);
    const size_t smem = 2 * (size_t)cap * sizeof(float4);
    if (smem <= kGradSmemMax) {
      CK(cudaFuncSetAttribute(k_grad_staged<kGradNB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
         "staged gradients");
      ctx->grad_cap = cap;
      ctx->grad_smem_attr = (int)smem;
    }
  }

  rt_status st;
#define AL(p, n) if ((st = dalloc(ctx, &(p), (n), #p))) return st
  AL(ctx->vol, C); AL(ctx->cx, C); AL(ctx->cy, C); AL(ctx->cz, C);
  AL(ctx->off, C + 1); AL(ctx->csr, 2 * (size_t)F); AL(ctx->nbr, 2 * (size_t)F); AL(ctx->lr, F);
  AL(ctx->nA64, F); AL(ctx->rL64, F); AL(ctx->rR64, F); AL(ctx->w64, F); AL(ctx->minv64, 6 * (size_t)C);
  if (ctx->cfg.time_order == 2) AL(ctx->rad0, (size_t)C * B);
  AL(ctx->rad, (size_t)C * B); AL(ctx->nH, C); AL(ctx->x5, 5 * (size_t)C); AL(ctx->T, C);
  AL(ctx->src_idx, C); AL(ctx->nsub, C); AL(ctx->status, 1);
  ctx->stage_n = std::max<size_t>(4 * (size_t)B * C, 7 * (size_t)F);
  ctx->stage_n = std::max<size_t>(ctx->stage_n, 5 * (size_t)C);
  AL(ctx->stage, ctx->stage_n);
  const bool mx = mixed(ctx);
  const size_t rs = mx ? 4 : 8;
  {
    void* p;
    const size_t gbytes = mx ? (size_t)C * 4 * pad_bins(B) * sizeof(float4) : (size_t)C * B * 12 * sizeof(double);
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(gbytes, 1));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "G");
    ctx->allocs.push_back(p); ctx->G = p;
    e = cudaMalloc(&p, std::max<size_t>((size_t)F * B * 4 * rs, 1));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "flux");
    ctx->allocs.push_back(p); ctx->flux = p;
    for (void** h : {&ctx->hw, &ctx->hx}) {
      e = cudaMalloc(&p, std::max<size_t>(2 * (size_t)F * 4 * rs, 1));
      if (e != cudaSuccess) return cuda_fail(ctx, e, "half-edges");
      ctx->allocs.push_back(p); *h = p;
    }
    e = cudaMalloc(&p, std::max<size_t>((size_t)C * rs, 1));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "half-edges");
    ctx->allocs.push_back(p); ctx->xmax = p;
  }
  AL(ctx->work_cell, C); AL(ctx->work_ctl, 4);
  if (mx) {
    AL(ctx->fa32, F); AL(ctx->fb32, F); AL(ctx->minv32, 6 * (size_t)C); AL(ctx->ivol, C);
    AL(ctx->work_f1, C);
    AL(ctx->shadow, (size_t)C * B);
    AL(ctx->radN, (size_t)C * B);
  } else {
    AL(ctx->work_f1d, C);
  }
#undef AL
  if ((st = copy_in(ctx, ctx->vol, cells->volume, (size_t)C * 8))) return st;
  if ((st = copy_in(ctx, ctx->cx, cells->cx, (size_t)C * 8))) return st;
  if ((st = copy_in(ctx, ctx->cy, cells->cy, (size_t)C * 8))) return st;
  if ((st = copy_in(ctx, ctx->cz, cells->cz, (size_t)C * 8))) return st;
  CK(cudaMemcpyAsync(ctx->off, off.data(), (C + 1) * 4, cudaMemcpyHostToDevice, ctx->stream), "off");
  CK(cudaMemcpyAsync(ctx->csr, csr.data(), 2 * (size_t)F * 4, cudaMemcpyHostToDevice, ctx->stream), "csr");
  CK(cudaMemcpyAsync(ctx->nbr, nbr.data(), 2 * (size_t)F * 4, cudaMemcpyHostToDevice, ctx->stream), "nbr");
  {
    std::vector<int2> lr(F);
    for (int f = 0; f < F; ++f) lr[f] = make_int2(L[f], Rr[f]);
    CK(cudaMemcpyAsync(ctx->lr, lr.data(), (size_t)F * 8, cudaMemcpyHostToDevice, ctx->stream), "lr");
    CK(cudaStreamSynchronize(ctx->stream), "mesh upload");
  }
  // face arrays through the staging buffer: area, n, x_f
  double* sA = ctx->stage;
  double *snx = sA + F, *sny = sA + 2 * (size_t)F, *snz = sA + 3 * (size_t)F;
  double *sfx = sA + 4 * (size_t)F, *sfy = sA + 5 * (size_t)F, *sfz = sA + 6 * (size_t)F;
  if (F > 0) {
    if ((st = copy_in(ctx, sA, faces->area, (size_t)F * 8))) return st;
    if ((st = copy_in(ctx, snx, faces->nx, (size_t)F * 8))) return st;
    if ((st = copy_in(ctx, sny, faces->ny, (size_t)F * 8))) return st;
    if ((st = copy_in(ctx, snz, faces->nz, (size_t)F * 8))) return st;
    if ((st = copy_in(ctx, sfx, faces->fx, (size_t)F * 8))) return st;
    if ((st = copy_in(ctx, sfy, faces->fy, (size_t)F * 8))) return st;
    if ((st = copy_in(ctx, sfz, faces->fz, (size_t)F * 8))) return st;
    k_pack_nA<<<nblk(F), kThreads, 0, ctx->stream>>>(F, snx, sny, snz, sA, ctx->nA64);
    k_geometry_faces<<<nblk(F), kThreads, 0, ctx->stream>>>(F, ctx->cfg.box, ctx->lr, ctx->cx, ctx->cy, ctx->cz,
                                                            sfx, sfy, sfz, sA, ctx->rL64, ctx->rR64, ctx->w64);
  }
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream), "status");
  CK(cudaMemsetAsync(ctx->work_ctl, 0, 4 * sizeof(int), ctx->stream), "worklist");
  k_geometry_cells<<<nblk(C), kThreads, 0, ctx->stream>>>(C, ctx->cfg.box, ctx->off, ctx->csr, ctx->lr, ctx->cx,
                                                          ctx->cy, ctx->cz, sA, ctx->minv64, ctx->status);
  if (mx && F > 0) {
    k_build_facerecs<<<nblk(F), kThreads, 0, ctx->stream>>>(F, ctx->lr, ctx->nA64, ctx->rL64, ctx->rR64, ctx->fa32,
                                                            ctx->fb32);
  }
  if (mx) {
    k_convert<float><<<nblk(6LL * C), kThreads, 0, ctx->stream>>>(6 * C, ctx->minv64, ctx->minv32);
    k_reciprocal<<<nblk(C), kThreads, 0, ctx->stream>>>(C, ctx->vol, ctx->ivol);
  }
  if (F > 0) {
    if (mx)
      k_build_halfedges<float><<<nblk(2LL * F), kThreads, 0, ctx->stream>>>(
          2 * F, ctx->csr, ctx->nbr, ctx->w64, ctx->rL64, ctx->rR64, (float4*)ctx->hw, (float4*)ctx->hx);
    else
      k_build_halfedges<double><<<nblk(2LL * F), kThreads, 0, ctx->stream>>>(
          2 * F, ctx->csr, ctx->nbr, ctx->w64, ctx->rL64, ctx->rR64, (d4*)ctx->hw, (d4*)ctx->hx);
    if (mx)
      k_cell_xmax<float><<<nblk(C), kThreads, 0, ctx->stream>>>(C, ctx->off, (const float4*)ctx->hx,
                                                               (float*)ctx->xmax);
    else
      k_cell_xmax<double><<<nblk(C), kThreads, 0, ctx->stream>>>(C, ctx->off, (const d4*)ctx->hx, (double*)ctx->xmax);
  }
  if ((st = launched(ctx, "geometry kernels"))) return st;
  int h_status = 0;
  CK(cudaMemcpyAsync(&h_status, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "status");
  CK(cudaStreamSynchronize(ctx->stream), "geometry");
  if (h_status & kStSingular) return fail(ctx, RT_BAD_MESH, "singular least-squares matrix (degenerate cell)");
  // default state: no radiation, neutral gas at 1e4 K, no sources
  CK(cudaMemsetAsync(ctx->rad, 0, (size_t)C * B * sizeof(d4), ctx->stream), "state");
  CK(cudaMemsetAsync(ctx->nH, 0, (size_t)C * 8, ctx->stream), "state");
  CK(cudaMemsetAsync(ctx->nsub, 0, (size_t)C * 4, ctx->stream), "state");
  CK(cudaMemsetAsync(ctx->src_idx, 0xff, (size_t)C * 4, ctx->stream), "state");
  {
    std::vector<double> x(5 * (size_t)C, 0.0), T(C, 1e4);
    std::fill(x.begin(), x.begin() + C, 1.0);
    std::fill(x.begin() + 2 * (size_t)C, x.begin() + 3 * (size_t)C, 1.0);
    CK(cudaMemcpyAsync(ctx->x5, x.data(), x.size() * 8, cudaMemcpyHostToDevice, ctx->stream), "state");
    CK(cudaMemcpyAsync(ctx->T, T.data(), T.size() * 8, cudaMemcpyHostToDevice, ctx->stream), "state");
    CK(cudaStreamSynchronize(ctx->stream), "state");
  }
  ctx->n_src_cells = 0;
  refresh_shadow(ctx);
  if ((st = launched(ctx, "state init"))) return st;
  ctx->mesh_ready = true;
  return RT_OK;
}

rt_status rt_set_gas(rt_ctx* ctx, const double* nH, const double* x5, const double* T) {
  rt_status st = need_mesh(ctx);
  if (st) return st;
  if (!nH || !x5 || !T) return fail(ctx, RT_INVALID_ARG, "gas array is NULL");
  const size_t C = ctx->C;
  if ((st = copy_in(ctx, ctx->nH, nH, C * 8))) return st;
  if ((st = copy_in(ctx, ctx->x5, x5, 5 * C * 8))) return st;
  if ((st = copy_in(ctx, ctx->T, T, C * 8))) return st;
  return RT_OK;
}

rt_status rt_set_radiation(rt_ctx* ctx, const double* N, const double* F) {
  rt_status st = need_mesh(ctx);
  if (st) return st;
  if (!N) return fail(ctx, RT_INVALID_ARG, "N is NULL");
  const size_t C = ctx->C, B = ctx->B;
  double* sN = ctx->stage;
  double* sF = ctx->stage + B * C;
  if ((st = copy_in(ctx, sN, N, B * C * 8))) return st;
  if (F && (st = copy_in(ctx, sF, F, 3 * B * C * 8))) return st;
  k_pack_rad<<<nblk((long long)B * C), kThreads, 0, ctx->stream>>>((int)C, (int)B, 1.0 / ctx->cfg.c_red, sN,
                                                                   F ? sF : nullptr, ctx->rad);
  refresh_shadow(ctx);
  return launched(ctx, "set radiation");
}

rt_status rt_set_sources(rt_ctx* ctx, int64_t n, const int64_t* cell, const double* Q) {
  rt_status st = need_mesh(ctx);
  if (st) return st;
  if (n < 0 || (n > 0 && (!cell || !Q))) return fail(ctx, RT_INVALID_ARG, "bad source arrays");
  const int B = ctx->B;
  std::vector<int64_t> hc(n);
  std::vector<double> hq((size_t)n * B);
  if (n > 0) {
    CK(cudaMemcpy(hc.data(), cell, n * 8, is_device_ptr(cell) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost),
       "sources");
    CK(cudaMemcpy(hq.data(), Q, n * B * 8, is_device_ptr(Q) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost),
       "sources");
  }
  // bin rates per cell, summed in source order
  std::vector<int32_t> idx(ctx->C, -1);
  std::vector<double> rate;
  int m = 0;
  for (int64_t k = 0; k < n; ++k) {
    if (hc[k] < 0 || hc[k] >= ctx->C) return fail(ctx, RT_INVALID_ARG, "source %lld in cell %lld out of range",
                                                  (long long)k, (long long)hc[k]);
    int32_t& s = idx[hc[k]];
    if (s < 0) {
      s = m++;
      rate.resize((size_t)m * B, 0.0);
    }
    for (int b = 0; b < B; ++b) rate[(size_t)s * B + b] += hq[(size_t)k * B + b];
  }
  if (m > ctx->src_cap) {
    double* p = nullptr;
    if ((st = dalloc(ctx, &p, (size_t)m * B, "source rates"))) return st;
    ctx->src_rate = p;
    ctx->src_cap = m;
  }
  CK(cudaMemcpyAsync(ctx->src_idx, idx.data(), (size_t)ctx->C * 4, cudaMemcpyHostToDevice, ctx->stream),
     "sources");
  if (m > 0)
    CK(cudaMemcpyAsync(ctx->src_rate, rate.data(), (size_t)m * B * 8, cudaMemcpyHostToDevice, ctx->stream),
       "sources");
  CK(cudaStreamSynchronize(ctx->stream), "sources");
  ctx->gen++;   // the source pointer and count are launch arguments
  ctx->n_src_cells = m;
  ctx->src_cells.assign(hc.begin(), hc.end());
  return RT_OK;
}

rt_status rt_max_dt(rt_ctx* ctx, double* out) {
  rt_status st = need_mesh(ctx);
  if (st) return st;
  if (!out) return fail(ctx, RT_INVALID_ARG, "out is NULL");
  *out = ctx->cfg.cfl * ctx->min_dx_cm / ctx->cfg.c_red;
  return RT_OK;
}

rt_status rt_mesh_info(rt_ctx* ctx, int64_t* n_cells, int64_t* n_faces, int32_t* max_degree) {
  rt_status st = need_mesh(ctx);
  if (st) return st;
  if (n_cells) *n_cells = ctx->C;
  if (n_faces) *n_faces = ctx->F;
  if (max_degree) *max_degree = ctx->max_deg;
  return RT_OK;
}

rt_status rt_set_active(rt_ctx* ctx, const uint8_t* active) {
  rt_status st = need_mesh(ctx);
  if (st) return st;
  // the lists may be in use by work already enqueued
  CK(cudaStreamSynchronize(ctx->stream), "rt_set_active");
  const int C = ctx->C, F = ctx->F, B = ctx->B;
  const int prev = ctx->cur_set;
  std::vector<uint8_t> m;
  bool all = true;
  if (active) {
    m.resize(C);
    CK(cudaMemcpy(m.data(), active, (size_t)C, is_device_ptr(active) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost),
       "active mask");
    for (int i = 0; i < C; ++i) {
      m[i] = m[i] != 0;
      all = all && m[i];
    }
  }
  if (all) {
    use_set(ctx, -1);
    return RT_OK;
  }
  // a mask seen recently keeps its lists and its step graph
  uint64_t h = 1469598103934665603ull;   // FNV-1a
  for (uint8_t v : m) h = (h ^ v) * 1099511628211ull;
  int k = -1;
  for (int j = 0; j < rt_ctx::kMaxActSets && k < 0; ++j)
    if (ctx->sets[j].valid && ctx->sets[j].hash == h && ctx->sets[j].mask == m) k = j;
  if (k < 0) {
    // a free slot, else the least recently used one
    for (int j = 0; j < rt_ctx::kMaxActSets && k < 0; ++j)
      if (!ctx->sets[j].valid) k = j;
    if (k < 0) {
      k = 0;
      for (int j = 1; j < rt_ctx::kMaxActSets; ++j)
        if (ctx->sets[j].used < ctx->sets[k].used) k = j;
    }
    rt_ctx::ActSet& a = ctx->sets[k];
    free_set(a);
    std::vector<int2> lr(F);
    if (F > 0) CK(cudaMemcpy(lr.data(), ctx->lr, (size_t)F * sizeof(int2), cudaMemcpyDeviceToHost), "active mask");
    std::vector<int32_t> ac, tc, af, gb;
    std::vector<uint8_t> tf(C, 0);
    for (int i = 0; i < C; ++i)
      if (m[i]) ac.push_back(i);
    for (int f = 0; f < F; ++f)
      if (m[lr[f].x] || m[lr[f].y]) {
        af.push_back(f);
        tf[lr[f].x] = tf[lr[f].y] = 1;
      }
    for (int i = 0; i < C; ++i)
      if (tf[i]) tc.push_back(i);
    for (int c0 = 0; c0 < C; c0 += kGradCells) {
      bool any = false;
      for (int i = c0; i < std::min(c0 + kGradCells, C) && !any; ++i) any = tf[i];
      if (any) gb.push_back(c0 / kGradCells);
    }
    // staged gradients over the touched list: the face records of the
    // largest block of kGradCells list entries must fit in shared memory
    int cap_list = 0;
    if (mixed(ctx) && ctx->grad_cap > 0) {
      std::vector<int32_t> deg(C, 0);
      for (int f = 0; f < F; ++f) {
        deg[lr[f].x]++;
        deg[lr[f].y]++;
      }
      for (size_t j0 = 0; j0 < tc.size(); j0 += kGradCells) {
        int sum = 0;
        for (size_t j = j0; j < std::min(j0 + kGradCells, tc.size()); ++j) sum += deg[tc[j]];
        cap_list = std::max(cap_list, sum);
      }
      const size_t smem = 2 * (size_t)cap_list * sizeof(float4);
      if (smem > kGradSmemMax) {
        cap_list = 0;
      } else if ((int)smem > ctx->grad_smem_attr) {
        CK(cudaFuncSetAttribute(k_grad_staged<kGradNB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
           "staged gradients");
        ctx->grad_smem_attr = (int)smem;
      }
    }
    auto up = [&](const void* src, size_t bytes, void** dst) -> rt_status {
      void* p = nullptr;
      cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
      if (e != cudaSuccess) return cuda_fail(ctx, e, "active lists");
      a.allocs.push_back(p);
      if (bytes) {
        e = cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "active lists");
      }
      *dst = p;
      return RT_OK;
    };
    if ((st = up(ac.data(), ac.size() * 4, (void**)&a.act_cells)) ||
        (st = up(tc.data(), tc.size() * 4, (void**)&a.touched_cells)) ||
        (st = up(af.data(), af.size() * 4, (void**)&a.act_faces)) ||
        (st = up(gb.data(), gb.size() * 4, (void**)&a.grad_blocks)) ||
        (st = up(tf.data(), tf.size(), (void**)&a.touched))) {
      free_set(a);
      use_set(ctx, -1);
      return st;
    }
    a.n_act = (int)ac.size();
    a.n_touched = (int)tc.size();
    a.n_act_faces = (int)af.size();
    a.n_grad_blocks = (int)gb.size();
    a.grad_cap_list = cap_list;
    a.hash = h;
    a.mask.swap(m);
    a.valid = true;
  }
  use_set(ctx, k);
  if (k != prev) {
    // the face kernel writes the active interfaces only: the others must
    // carry no flux while this set holds
    const size_t rs = mixed(ctx) ? 4 : 8;
    CK(cudaMemsetAsync(ctx->flux, 0, (size_t)F * B * 4 * rs, ctx->stream), "active mask");
  }
  return RT_OK;
}

rt_status rt_step(rt_ctx* ctx, double dt, int n_sub) {
  rt_status st = need_mesh(ctx);
  if (st) return st;
  if (n_sub < 1 || !(dt > 0) || !std::isfinite(dt)) return fail(ctx, RT_INVALID_ARG, "need dt > 0 and n_sub >= 1");
  const double dts = dt / n_sub;
  const double dmax = ctx->cfg.cfl * ctx->min_dx_cm / ctx->cfg.c_red;
  if (dts > dmax * (1.0 + 1e-12))
    return fail(ctx, RT_CFL, "subcycle %g s exceeds the CFL limit %g s", dts, dmax);
  // Replay the captured graph of this step if nothing it depends on changed.
  rt_ctx::GraphSlot& g = cur_graph(ctx);
  if (g.exec && g.gen == ctx->gen && g.dt == dt && g.nsub == n_sub && !ctx->profiling) {
    CK(cudaGraphLaunch(g.exec, ctx->stream), "rt_step graph");
    ctx->launches += g.launches;
    return RT_OK;
  }
  // Otherwise capture the step's launches into a graph -- on an internal
  // stream, so that any stream of the caller (the legacy default included)
  // can replay it -- and launch it.  Not while profiling with events, nor
  // when the caller's stream is itself being captured (the launches then
  // become part of the caller's graph).
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  bool capture = !ctx->profiling && cudaStreamIsCapturing(ctx->stream, &cs) == cudaSuccess &&
                 cs == cudaStreamCaptureStatusNone;
  cudaGetLastError();
  if (capture && !ctx->cap_stream &&
      cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    ctx->cap_stream = nullptr;
    capture = false;
  }
  cudaStream_t user = ctx->stream;
  if (capture) {
    drop_graph(g);
    ctx->stream = ctx->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      ctx->stream = user;
      return cuda_fail(ctx, e, "rt_step capture");
    }
  }
  const int64_t l0 = ctx->launches;
  // Subcycle: sources + chemistry, gradients, fluxes, application (Lie);
  // Strang puts half the chemistry on each side of the transport.
  const bool strang = ctx->cfg.splitting == 1;
  for (int s = 0; s < n_sub; ++s) {
    launch_chem(ctx, strang ? 0.5 * dts : dts);
    transport(ctx, dts);
    if (strang) launch_chem(ctx, 0.5 * dts);
  }
  if (!capture) return launched(ctx, "rt_step");
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
  ctx->stream = user;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "rt_step capture");
  e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g.exec = nullptr;
    return cuda_fail(ctx, e, "rt_step graph");
  }
  g.gen = ctx->gen;
  g.dt = dt;
  g.nsub = n_sub;
  g.launches = ctx->launches - l0;
  CK(cudaGraphLaunch(g.exec, ctx->stream), "rt_step graph");
  return RT_OK;
}

rt_status rt_sync(rt_ctx* ctx) {
  rt_status st = need_mesh(ctx);
  if (st) return st;
  int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "status");
  CK(cudaStreamSynchronize(ctx->stream), "rt_sync");
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream), "status");
  if (h & kStTimeout) return fail(ctx, RT_TIMEOUT, "a device wait for a bulk copy gave up");
  if (h & kStNonFinite) return fail(ctx, RT_NONFINITE, "non-finite photon density");
  if (h & kStChemSubsteps) return fail(ctx, RT_CHEM_SUBSTEPS, "a cell reached max_substeps");
  return RT_OK;
}

rt_status rt_get_fields(rt_ctx* ctx, uint32_t mask, double* const* out) {
  rt_status st = need_mesh(ctx);
  if (st) return st;
  if (!out && mask) return fail(ctx, RT_INVALID_ARG, "out is NULL");
  const size_t C = ctx->C, B = ctx->B;
  int k = 0;
  if (mask & (RT_FIELD_N | RT_FIELD_F)) {
    double* sN = ctx->stage;
    double* sF = ctx->stage + B * C;
    join_state(ctx);
    k_unpack_rad<<<nblk((long long)B * C), kThreads, 0, ctx->stream>>>((int)C, (int)B, ctx->cfg.c_red, ctx->rad,
                                                                        sN, sF);
    if ((st = launched(ctx, "get fields"))) return st;
    if (mask & RT_FIELD_N) {
      if (!out[k]) return fail(ctx, RT_INVALID_ARG, "output %d is NULL", k);
      if ((st = copy_out(ctx, out[k++], sN, B * C * 8))) return st;
    }
    if (mask & RT_FIELD_F) {
      if (!out[k]) return fail(ctx, RT_INVALID_ARG, "output %d is NULL", k);
      if ((st = copy_out(ctx, out[k++], sF, 3 * B * C * 8))) return st;
    }
  }
  if (mask & RT_FIELD_X) {
    if (!out[k]) return fail(ctx, RT_INVALID_ARG, "output %d is NULL", k);
    if ((st = copy_out(ctx, out[k++], ctx->x5, 5 * C * 8))) return st;
  }
  if (mask & RT_FIELD_T) {
    if (!out[k]) return fail(ctx, RT_INVALID_ARG, "output %d is NULL", k);
    if ((st = copy_out(ctx, out[k++], ctx->T, C * 8))) return st;
  }
  if (mask & RT_FIELD_NSUB) {
    if (!out[k]) return fail(ctx, RT_INVALID_ARG, "output %d is NULL", k);
    std::vector<int32_t> h(C);
    CK(cudaMemcpyAsync(h.data(), ctx->nsub, C * 4, cudaMemcpyDeviceToHost, ctx->stream), "nsub");
    CK(cudaStreamSynchronize(ctx->stream), "nsub");
    std::vector<double> d(h.begin(), h.end());
    if ((st = copy_in(ctx, ctx->stage, d.data(), C * 8))) return st;
    if ((st = copy_out(ctx, out[k++], ctx->stage, C * 8))) return st;
  }
  CK(cudaStreamSynchronize(ctx->stream), "get fields");
  return RT_OK;
}

// ---- stage entry points -----------------------------------------------------

rt_status rt_stage_gradients(rt_ctx* ctx, double* G) {
  rt_status st = need_mesh(ctx);
  if (st) return st;
  launch_grad_any(ctx);
  if ((st = launched(ctx, "gradients"))) return st;
  if (!G) return RT_OK;
  const size_t n = (size_t)ctx->C * ctx->B * 12;
  if (mixed(ctx)) {
    // widen the gradient groups of the cell-major records in a host buffer
    const int Bp = pad_bins(ctx->B);
    std::vector<float4> h((size_t)ctx->C * 4 * Bp);
    CK(cudaMemcpyAsync(h.data(), ctx->G, h.size() * sizeof(float4), cudaMemcpyDeviceToHost, ctx->stream),
       "gradients");
    CK(cudaStreamSynchronize(ctx->stream), "gradients");
    std::vector<double> d(n);
    for (int i = 0; i < ctx->C; ++i)
      for (int b = 0; b < ctx->B; ++b)
        for (int v = 0; v < 3; ++v) {
          const float4 q = h[grec(i, v, b, Bp)];
          double* o = d.data() + ((size_t)i * ctx->B + b) * 12 + 4 * v;
          o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
        }
    if (is_device_ptr(G)) {
      CK(cudaMemcpy(G, d.data(), n * 8, cudaMemcpyHostToDevice), "gradients");
    } else {
      std::memcpy(G, d.data(), n * 8);
    }
    return RT_OK;
  }
  return copy_out(ctx, G, ctx->G, n * 8);
}

rt_status rt_stage_fluxes(rt_ctx* ctx, const double* G, double* flux) {
  rt_status st = need_mesh(ctx);
  if (st) return st;
  const size_t nG = (size_t)ctx->C * ctx->B * 12, nF = (size_t)ctx->F * ctx->B * 4;
  if (G) {
    if (mixed(ctx)) {
      // cell-major records: the given gradients, then the FP32 cell state
      const size_t nr = (size_t)ctx->C * ctx->B;
      const int Bp = pad_bins(ctx->B);
      std::vector<double> d(nG);
      CK(cudaMemcpy(d.data(), G, nG * 8, is_device_ptr(G) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost), "G");
      std::vector<float4> sh(nr);
      CK(cudaMemcpy(sh.data(), ctx->shadow, nr * sizeof(float4), cudaMemcpyDeviceToHost), "G");
      std::vector<float4> h((size_t)ctx->C * 4 * Bp, make_float4(0.f, 0.f, 0.f, 0.f));
      for (int i = 0; i < ctx->C; ++i)
        for (int b = 0; b < ctx->B; ++b) {
          const double* q = d.data() + ((size_t)i * ctx->B + b) * 12;
          for (int v = 0; v < 3; ++v)
            h[grec(i, v, b, Bp)] = make_float4((float)q[4 * v], (float)q[4 * v + 1], (float)q[4 * v + 2],
                                               (float)q[4 * v + 3]);
          h[grec(i, 3, b, Bp)] = sh[(size_t)i * ctx->B + b];
        }
      CK(cudaMemcpy(ctx->G, h.data(), h.size() * sizeof(float4), cudaMemcpyHostToDevice), "G");
    } else if ((st = copy_in(ctx, ctx->G, G, nG * 8))) {
      return st;
    }
  } else {
    launch_grad_any(ctx);
  }
  launch_flux_any(ctx);
  if ((st = launched(ctx, "fluxes"))) return st;
  if (!flux) return RT_OK;
  if (mixed(ctx)) {
    std::vector<float> h(nF);
    CK(cudaMemcpyAsync(h.data(), ctx->flux, nF * 4, cudaMemcpyDeviceToHost, ctx->stream), "fluxes");
    CK(cudaStreamSynchronize(ctx->stream), "fluxes");
    std::vector<double> d(h.begin(), h.end());
    if (is_device_ptr(flux)) CK(cudaMemcpy(flux, d.data(), nF * 8, cudaMemcpyHostToDevice), "fluxes");
    else std::memcpy(flux, d.data(), nF * 8);
    return RT_OK;
  }
  return copy_out(ctx, flux, ctx->flux, nF * 8);
}

rt_status rt_stage_transport(rt_ctx* ctx, double dt) {
  rt_status st = need_mesh(ctx);
  if (st) return st;
  if (!(dt >= 0)) return fail(ctx, RT_INVALID_ARG, "dt must be >= 0");
  transport(ctx, dt);
  return launched(ctx, "transport");
}

rt_status rt_stage_chemistry(rt_ctx* ctx, double dt) {
  rt_status st = need_mesh(ctx);
  if (st) return st;
  if (!(dt >= 0)) return fail(ctx, RT_INVALID_ARG, "dt must be >= 0");
  launch_chem(ctx, dt);
  return launched(ctx, "chemistry");
}

rt_status rt_profile_enable(rt_ctx* ctx, int on) {
  if (!ctx) return fail(nullptr, RT_INVALID_ARG, "null context");
  ctx->profiling = on != 0;
  return RT_OK;
}

rt_status rt_profile_read(rt_ctx* ctx, int n, double* ms, int64_t* launches, int reset) {
  if (!ctx) return fail(nullptr, RT_INVALID_ARG, "null context");
  CK(cudaStreamSynchronize(ctx->stream), "profile");
  for (auto& u : ctx->ev_used) {
    float t = 0;
    CK(cudaEventElapsedTime(&t, ctx->ev_pool[u.second], ctx->ev_pool[u.second + 1]), "profile");
    ctx->prof_ms[u.first] += t;
    ctx->prof_n[u.first] += 1;
  }
  ctx->ev_used.clear();
  for (int k = 0; k < n && k < RT_KERNEL_COUNT; ++k) {
    if (ms) ms[k] = ctx->prof_ms[k];
    if (launches) launches[k] = ctx->prof_n[k];
  }
  if (reset)
    for (int k = 0; k < RT_KERNEL_COUNT; ++k) { ctx->prof_ms[k] = 0; ctx->prof_n[k] = 0; }
  return RT_OK;
}

rt_status rt_launch_count(rt_ctx* ctx, int64_t* out) {
  if (!ctx || !out) return fail(ctx, RT_INVALID_ARG, "null argument");
  *out = ctx->launches;
  return RT_OK;
}

}  // extern "C"

// ---- adjoint ------------------------------------------------------------------

namespace {

template <class T> rt_status aalloc(rt_ctx* ctx, T** p, size_t n, const char* what) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  ctx->adj.allocs.push_back(q);
  *p = (T*)q;
  return RT_OK;
}

void adj_free(rt_ctx* ctx) {
  for (void* p : ctx->adj.allocs) cudaFree(p);
  ctx->adj = rt_ctx::Adj();
}

// The chemistry tape: room for `want` records (at least `need`, should
// `want` not fit in device memory), keeping the first `keep`.
rt_status tape_grow(rt_ctx* ctx, long long want, long long need, long long keep) {
  auto& A = ctx->adj;
  if (need <= A.rec_cap) return RT_OK;
  if (need > 0x7fffffffLL) return fail(ctx, RT_OOM, "adjoint: a segment's chemistry tape exceeds 2^31 attempts");
  long long n = std::min<long long>(std::max(want, need), 0x7fffffffLL);
  ChemRec* r = nullptr;
  rt_status st = aalloc(ctx, &r, (size_t)n, "chemistry tape");
  if (st && n > need) {
    cudaGetLastError();   // an allocation failure is not sticky: try the exact need
    n = need;
    st = aalloc(ctx, &r, (size_t)n, "chemistry tape");
  }
  if (st) return st;
  if (A.rec) {
    if (keep > 0)
      CK(cudaMemcpyAsync(r, A.rec, (size_t)keep * sizeof(ChemRec), cudaMemcpyDeviceToDevice, ctx->stream), "tape");
    CK(cudaStreamSynchronize(ctx->stream), "tape");
    cudaFree(A.rec);
    A.allocs.erase(std::find(A.allocs.begin(), A.allocs.end(), A.rec));
  }
  A.rec = r;
  A.rec_cap = n;
  return RT_OK;
}

// Room for attempt_lin of n records.
rt_status lin_reserve(rt_ctx* ctx, long long n) {
  auto& A = ctx->adj;
  if (n <= A.lin_cap) return RT_OK;
  if (A.lin) {
    CK(cudaStreamSynchronize(ctx->stream), "tape");
    cudaFree(A.lin);
    A.allocs.erase(std::find(A.allocs.begin(), A.allocs.end(), A.lin));
    A.lin = nullptr;
    A.lin_cap = 0;
  }
  AttemptLin* l = nullptr;
  rt_status st = aalloc(ctx, &l, (size_t)n, "chemistry linearisation");
  if (st) return st;
  A.lin = l;
  A.lin_cap = n;
  return RT_OK;
}

rt_status adj_prepare(rt_ctx* ctx, int nseg, int k) {
  auto& A = ctx->adj;
  if (A.nseg >= nseg && A.k >= k && A.lam_rad) return RT_OK;
  adj_free(ctx);
  const size_t C = ctx->C, F = ctx->F, B = ctx->B;
  rt_status st;
#define AA(p, n) if ((st = aalloc(ctx, &(p), (n), #p))) return st
  // checkpoints of every segment but the last, which the forward records
  AA(A.ck_rad, (nseg - 1) * C * B); AA(A.ck_x5, (nseg - 1) * 5 * C); AA(A.ck_T, (nseg - 1) * C);
  AA(A.tp_rad_chem, k * C * B); AA(A.tp_rad_trans, k * C * B); AA(A.tp_x5, k * 5 * C); AA(A.tp_T, k * C);
  AA(A.fin_rad, C * B); AA(A.fin_x5, 5 * C); AA(A.fin_T, C);
  AA(A.lam_rad, C * B); AA(A.lam_part, C * B); AA(A.lam_in, C * B); AA(A.lampre, F * B * 2); AA(A.lamr, C * B * 3);
  AA(A.lam_x5, 5 * C); AA(A.lam_T, C); AA(A.lam_nH, C); AA(A.lam_S, B * C); AA(A.lim_coef, C * B * 4);
  AA(A.lim_cell, C * B * 4);
  AA(A.tape_last, (size_t)k * C); AA(A.tape_used, 1);
#undef AA
  const long long first = std::max<long long>(4096, (long long)C / 4);
  if ((st = tape_grow(ctx, first, first, 0))) return st;
  A.nseg = nseg;
  A.k = k;
  return RT_OK;
}

rt_status adj_copy_state(rt_ctx* ctx, d4* rad, double* x5, double* T, bool save) {
  const size_t C = ctx->C, B = ctx->B;
  cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
  if (save) {
    CK(cudaMemcpyAsync(rad, ctx->rad, C * B * sizeof(d4), k, ctx->stream), "checkpoint");
    CK(cudaMemcpyAsync(x5, ctx->x5, 5 * C * 8, k, ctx->stream), "checkpoint");
    CK(cudaMemcpyAsync(T, ctx->T, C * 8, k, ctx->stream), "checkpoint");
  } else {
    CK(cudaMemcpyAsync(ctx->rad, rad, C * B * sizeof(d4), k, ctx->stream), "restore");
    CK(cudaMemcpyAsync(ctx->x5, x5, 5 * C * 8, k, ctx->stream), "restore");
    CK(cudaMemcpyAsync(ctx->T, T, C * 8, k, ctx->stream), "restore");
  }
  return RT_OK;
}

AdjArgs adj_args(rt_ctx* ctx, const d4* rad, double dt) {
  AdjArgs a;
  a.C = ctx->C; a.F = ctx->F; a.B = ctx->B; a.off = ctx->off; a.csr = ctx->csr; a.nbr = ctx->nbr; a.lr = ctx->lr;
  a.nA = ctx->nA64; a.rL = ctx->rL64; a.rR = ctx->rR64; a.w = ctx->w64; a.minv = ctx->minv64; a.vol = ctx->vol;
  a.rad = rad; a.G = (const double*)ctx->G; a.lam_out = ctx->adj.lam_rad; a.lampre = ctx->adj.lampre;
  a.lamr = ctx->adj.lamr; a.lim_coef = ctx->adj.lim_coef; a.lim_cell = ctx->adj.lim_cell;
  a.lam_part = ctx->adj.lam_part; a.lam_in = ctx->adj.lam_in;
  a.lam = ctx->cfg.c_red * dt / ctx->cfg.unit_length_cm;
  a.order = ctx->cfg.order; a.limiter = ctx->cfg.limiter; a.lim_eps2 = ctx->cfg.lim_eps * ctx->cfg.lim_eps;
  return a;
}

ChemAdjArgs chem_adj_args(rt_ctx* ctx, const d4* rad, const double* x5, const double* T, double dt) {
  ChemAdjArgs a;
  a.C = ctx->C; a.B = ctx->B; a.rad = rad; a.x5 = x5; a.T = T; a.nH = ctx->nH; a.vol = ctx->vol;
  a.rec = (const ChemRec*)ctx->adj.rec; a.last = nullptr; a.lin = nullptr; a.rec_lo = a.rec_hi = 0;
  a.lam_rad = ctx->adj.lam_rad; a.lam_x5 = ctx->adj.lam_x5; a.lam_T = ctx->adj.lam_T; a.lam_nH = ctx->adj.lam_nH;
  a.lam_S = ctx->adj.lam_S; a.status = ctx->status; a.src_idx = ctx->src_idx; a.src_rate = ctx->src_rate;
  a.dt = dt;
  const double lu = ctx->cfg.unit_length_cm;
  a.lu3 = lu * lu * lu;
  a.do_inject = ctx->n_src_cells > 0;
  a.do_chem = ctx->cfg.chem_mode > 0;
  return a;
}

// Reverse of one subcycle: transport (from the recorded pre-transport
// radiation), then chemistry and sources (from the recorded pre-chemistry
// state and the recorded attempts).
rt_status adj_subcycle(rt_ctx* ctx, int slot, double dts) {
  auto& A = ctx->adj;
  const size_t C = ctx->C, B = ctx->B;
  const long long nCB = (long long)C * B, nFB = (long long)ctx->F * B;
  const d4* rt_rad = A.tp_rad_trans + slot * C * B;
  // gradients of the recorded state
  k_grad<double><<<nblk(nCB), kThreads, 0, ctx->stream>>>(
      geo<double>(ctx), rt_rad, (double*)ctx->G, ctx->cfg.order, ctx->cfg.limiter,
      ctx->cfg.lim_eps * ctx->cfg.lim_eps);
  AdjArgs a = adj_args(ctx, rt_rad, dts);
  k_adj_face<<<nblk(nFB), kThreads, 0, ctx->stream>>>(a);
  k_adj_cellgrad<<<nblk(nCB), kThreads, 0, ctx->stream>>>(a);
  k_adj_cellsum<<<nblk(nCB), kThreads, 0, ctx->stream>>>(a);
  std::swap(A.lam_rad, A.lam_in);
  rt_status st = launched(ctx, "adjoint transport");
  if (st) return st;
  // chemistry, from the records of the segment's recompute
  const d4* pc_rad = A.tp_rad_chem + slot * C * B;
  const double* pc_x5 = A.tp_x5 + slot * 5 * C;
  const double* pc_T = A.tp_T + slot * C;
  ChemParams P = chem_params(ctx);
  ChemAdjArgs ca = chem_adj_args(ctx, pc_rad, pc_x5, pc_T, dts);
  ca.last = A.tape_last + (size_t)slot * C;
  ca.lin = (const AttemptLin*)A.lin;
  ca.rec_lo = A.slot_rec[slot];
  ca.rec_hi = A.slot_rec[slot + 1];
  const int t = 128;
  const long long nrec = ca.rec_hi - ca.rec_lo;
  switch (B) {
#define CHEM_ADJ(KB)                                                                                      \
  case KB:                                                                                                \
    if (nrec > 0) k_chem_lin<KB><<<nblk(nrec, t), t, 0, ctx->stream>>>(ca, P, (AttemptLin*)A.lin);        \
    k_chem_adj<KB><<<nblk(C, t), t, 0, ctx->stream>>>(ca, P);                                             \
    break;
    CHEM_ADJ(1)
    CHEM_ADJ(2)
    CHEM_ADJ(3)
#undef CHEM_ADJ
    default:
      return fail(ctx, RT_INVALID_ARG, "adjoint: %d bins", (int)B);
  }
  return launched(ctx, "adjoint chemistry");
}

// Run the subcycles [s0, s1) of a segment forward from the context's state
// and record them for the reverse mode: the states entering each subcycle's
// chemistry and transport, and the worklist's chemistry attempts.  The
// transport of the segment's last subcycle runs only if `finish` (the
// forward pass needs the end state, a recompute does not).  The host reads
// the record counter after each subcycle's chemistry (the subcycle's range
// of records); should the tape have overflowed, it grows, keeping the
// earlier subcycles' records, and that subcycle's chemistry runs again
// from its recorded entering state.
rt_status adj_record_segment(rt_ctx* ctx, int s0, int s1, double dts, bool finish) {
  auto& A = ctx->adj;
  const size_t C = ctx->C, B = ctx->B;
  const bool chem = ctx->cfg.chem_mode > 0;
  const cudaMemcpyKind d2d = cudaMemcpyDeviceToDevice;
  A.slot_rec.assign(s1 - s0 + 1, 0);
  CK(cudaMemsetAsync(A.tape_used, 0, sizeof(unsigned long long), ctx->stream), "tape");
  CK(cudaMemsetAsync(A.tape_last, 0xff, (size_t)(s1 - s0) * C * sizeof(int32_t), ctx->stream), "tape");
  long long widest = 0;
  for (int s = s0; s < s1; ++s) {
    const int slot = s - s0;
    d4* r_chem = A.tp_rad_chem + slot * C * B;
    double* x_chem = A.tp_x5 + slot * 5 * C;
    double* T_chem = A.tp_T + slot * C;
    CK(cudaMemcpyAsync(r_chem, ctx->rad, C * B * sizeof(d4), d2d, ctx->stream), "tape");
    CK(cudaMemcpyAsync(x_chem, ctx->x5, 5 * C * 8, d2d, ctx->stream), "tape");
    CK(cudaMemcpyAsync(T_chem, ctx->T, C * 8, d2d, ctx->stream), "tape");
    long long used = A.slot_rec[slot];
    for (int tries = 0;; ++tries) {
      const ChemTape tape{(ChemRec*)A.rec, A.rec_cap, A.tape_used, A.tape_last + (size_t)slot * C};
      launch_chem(ctx, dts, chem ? &tape : nullptr);
      if (!chem) break;
      unsigned long long u = 0;
      CK(cudaMemcpyAsync(&u, A.tape_used, sizeof(u), cudaMemcpyDeviceToHost, ctx->stream), "tape");
      CK(cudaStreamSynchronize(ctx->stream), "tape");
      used = (long long)u;
      if (used <= A.rec_cap) break;
      if (tries > 0) return fail(ctx, RT_CUDA, "adjoint: a subcycle's chemistry tape does not repeat itself");
      rt_status st = tape_grow(ctx, std::max(2 * A.rec_cap, used + used / 4 + 1024), used, A.slot_rec[slot]);
      if (st) return st;
      const unsigned long long back = (unsigned long long)A.slot_rec[slot];
      CK(cudaMemcpyAsync(A.tape_used, &back, sizeof(back), cudaMemcpyHostToDevice, ctx->stream), "tape");
      CK(cudaMemsetAsync(A.tape_last + (size_t)slot * C, 0xff, C * sizeof(int32_t), ctx->stream), "tape");
      CK(cudaMemcpyAsync(ctx->rad, r_chem, C * B * sizeof(d4), d2d, ctx->stream), "tape");
      CK(cudaMemcpyAsync(ctx->x5, x_chem, 5 * C * 8, d2d, ctx->stream), "tape");
      CK(cudaMemcpyAsync(ctx->T, T_chem, C * 8, d2d, ctx->stream), "tape");
      CK(cudaStreamSynchronize(ctx->stream), "tape");   // `back` is read before it goes out of scope
      A.redone++;
    }
    A.slot_rec[slot + 1] = used;
    widest = std::max(widest, used - A.slot_rec[slot]);
    CK(cudaMemcpyAsync(A.tp_rad_trans + slot * C * B, ctx->rad, C * B * sizeof(d4), d2d, ctx->stream), "tape");
    if (s + 1 == s1 && !finish) break;
    launch_grad_any(ctx);
    launch_flux_any(ctx);
    launch_gather(ctx, dts);
  }
  A.tape_max = std::max(A.tape_max, A.slot_rec[s1 - s0]);
  rt_status st = lin_reserve(ctx, std::max<long long>(widest, 1));
  if (st) return st;
  return launched(ctx, "adjoint record");
}

}  // namespace

extern "C" {

rt_status rt_adjoint(rt_ctx* ctx, double dt, int n_sub, int checkpoint_every, const double* lam_N,
                     const double* lam_F, const double* lam_x5, const double* lam_T, double* dL_dQ,
                     double* dL_dnH, double* lam0_N, double* lam0_F, double* lam0_x5, double* lam0_T) {
  rt_status st = need_mesh(ctx);
  if (st) return st;
  if (mixed(ctx) || ctx->cfg.splitting != 0 || ctx->cfg.time_order != 1 || !ctx->all_active)
    return fail(ctx, RT_INVALID_ARG,
                "rt_adjoint supports FP64 precision, Lie splitting, forward-Euler transport, every cell active");
  if (n_sub < 1 || !(dt > 0) || !std::isfinite(dt) || checkpoint_every < 1)
    return fail(ctx, RT_INVALID_ARG, "need dt > 0, n_sub >= 1, checkpoint_every >= 1");
  const double dts = dt / n_sub;
  const double dmax = ctx->cfg.cfl * ctx->min_dx_cm / ctx->cfg.c_red;
  if (dts > dmax * (1.0 + 1e-12)) return fail(ctx, RT_CFL, "subcycle %g s exceeds the CFL limit %g s", dts, dmax);
  const int k = std::min(checkpoint_every, n_sub);
  const int nseg = (n_sub + k - 1) / k;
  if ((st = adj_prepare(ctx, nseg, k))) return st;
  auto& A = ctx->adj;
  const size_t C = ctx->C, B = ctx->B;
  A.tape_max = 0;
  A.redone = 0;
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream), "status");
  // forward with checkpoints; the last segment is recorded on the way
  const int s_last = (nseg - 1) * k;
  for (int s = 0; s < s_last; ++s) {
    if (s % k == 0 && (st = adj_copy_state(ctx, A.ck_rad + (s / k) * C * B, A.ck_x5 + (s / k) * 5 * C,
                                           A.ck_T + (s / k) * C, true)))
      return st;
    launch_chem(ctx, dts);
    launch_grad_any(ctx);
    launch_flux_any(ctx);
    launch_gather(ctx, dts);
  }
  if ((st = launched(ctx, "adjoint forward"))) return st;
  if ((st = adj_record_segment(ctx, s_last, n_sub, dts, true))) return st;
  if ((st = adj_copy_state(ctx, A.fin_rad, A.fin_x5, A.fin_T, true))) return st;
  // cotangents of the final state
  double* sN = ctx->stage;
  double* sF = ctx->stage + B * C;
  CK(cudaMemsetAsync(ctx->stage, 0, 4 * B * C * 8, ctx->stream), "adjoint");
  if (lam_N && (st = copy_in(ctx, sN, lam_N, B * C * 8))) return st;
  if (lam_F && (st = copy_in(ctx, sF, lam_F, 3 * B * C * 8))) return st;
  // dL/d(F/c) = c dL/dF
  k_pack_rad<<<nblk((long long)B * C), kThreads, 0, ctx->stream>>>((int)C, (int)B, ctx->cfg.c_red, sN, sF, A.lam_rad);
  CK(cudaMemsetAsync(A.lam_x5, 0, 5 * C * 8, ctx->stream), "adjoint");
  CK(cudaMemsetAsync(A.lam_T, 0, C * 8, ctx->stream), "adjoint");
  if (lam_x5 && (st = copy_in(ctx, A.lam_x5, lam_x5, 5 * C * 8))) return st;
  if (lam_T && (st = copy_in(ctx, A.lam_T, lam_T, C * 8))) return st;
  CK(cudaMemsetAsync(A.lam_nH, 0, C * 8, ctx->stream), "adjoint");
  CK(cudaMemsetAsync(A.lam_S, 0, B * C * 8, ctx->stream), "adjoint");
  // reverse, segment by segment; every segment but the last is recorded
  // again from its checkpoint
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int s0 = seg * k, s1 = std::min(n_sub, s0 + k);
    if (seg < nseg - 1) {
      if ((st = adj_copy_state(ctx, A.ck_rad + seg * C * B, A.ck_x5 + seg * 5 * C, A.ck_T + seg * C, false)))
        return st;
      if ((st = adj_record_segment(ctx, s0, s1, dts, false))) return st;
    }
    for (int s = s1 - 1; s >= s0; --s)
      if ((st = adj_subcycle(ctx, s - s0, dts))) return st;
  }
  if ((st = adj_copy_state(ctx, A.fin_rad, A.fin_x5, A.fin_T, false))) return st;
  // outputs
  if (dL_dQ && !ctx->src_cells.empty()) {
    std::vector<double> hS(B * C);
    CK(cudaMemcpyAsync(hS.data(), A.lam_S, B * C * 8, cudaMemcpyDeviceToHost, ctx->stream), "adjoint");
    CK(cudaStreamSynchronize(ctx->stream), "adjoint");
    std::vector<double> q(ctx->src_cells.size() * B);
    for (size_t s = 0; s < ctx->src_cells.size(); ++s)
      for (size_t b = 0; b < B; ++b) q[s * B + b] = hS[b * C + ctx->src_cells[s]];
    if (is_device_ptr(dL_dQ)) CK(cudaMemcpy(dL_dQ, q.data(), q.size() * 8, cudaMemcpyHostToDevice), "dL_dQ");
    else std::memcpy(dL_dQ, q.data(), q.size() * 8);
  }
  if (dL_dnH && (st = copy_out(ctx, dL_dnH, A.lam_nH, C * 8))) return st;
  if (lam0_N || lam0_F) {
    k_unpack_rad<<<nblk((long long)B * C), kThreads, 0, ctx->stream>>>((int)C, (int)B, 1.0 / ctx->cfg.c_red,
                                                                        A.lam_rad, sN, sF);
    if (lam0_N && (st = copy_out(ctx, lam0_N, sN, B * C * 8))) return st;
    if (lam0_F && (st = copy_out(ctx, lam0_F, sF, 3 * B * C * 8))) return st;
  }
  if (lam0_x5 && (st = copy_out(ctx, lam0_x5, A.lam_x5, 5 * C * 8))) return st;
  if (lam0_T && (st = copy_out(ctx, lam0_T, A.lam_T, C * 8))) return st;
  int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "status");
  CK(cudaStreamSynchronize(ctx->stream), "adjoint");
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream), "status");
  if (h & kStChemSubsteps) return fail(ctx, RT_CHEM_SUBSTEPS, "a cell reached max_substeps");
  if (h & kStNonFinite) return fail(ctx, RT_NONFINITE, "non-finite photon density");
  return launched(ctx, "adjoint");
}

rt_status rt_adjoint_tape_info(rt_ctx* ctx, long long* max_records, long long* capacity, int* redone) {
  if (!ctx) return fail(nullptr, RT_INVALID_ARG, "null context");
  if (max_records) *max_records = ctx->adj.tape_max;
  if (capacity) *capacity = ctx->adj.rec_cap;
  if (redone) *redone = ctx->adj.redone;
  return RT_OK;
}

const char* rt_last_error(const rt_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

void rt_destroy(rt_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  adj_free(ctx);
  free_all(ctx);
  delete ctx;
}

}  // extern "C"
