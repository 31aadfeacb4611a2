// bk_solve_batched and bk_autotune: many independent dense SPD systems of uneven size.
// Systems are grouped by padded block width; each group advances with one launch per
// step kernel (k_batch.cu), a chunk of steps replayed as a CUDA graph, and the host
// polls the per-system control blocks between chunks. FP64 refinement as in bk_solve.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "../../include/bk.h"
#include "bk_batch.cuh"
#include "bk_common.cuh"
#include "bk_ctx.h"

using namespace bkx;

namespace {

struct Group {
  int mp = 0;
  std::vector<int> members;  // indices into the caller's batch
  std::vector<bk::BSys> hs;  // host copies of the descriptors
  std::vector<int> hcta;     // thread-block -> local system table
  bk::BSys* ds = nullptr;    // device descriptors
  int* cta_sys = nullptr;    // device copy of hcta
  int ncta = 0;
  cudaGraphExec_t gexec = nullptr;
  // tensor-core block product (all systems of the group qualify); otherwise the FFMA
  // product with row tiles of tile_rows rows
  bool tc = false;
  int tile_rows = 16;
  std::vector<int> htile;        // tile_sys then tile_row
  std::vector<CUtensorMap> hmaps;  // two per system
  bk::BatchTc btc;
};

int size_bucket(int64_t d) {
  int b = 0;
  while ((int64_t)1 << (b + 1) <= d && b < 62) ++b;
  return b;  // floor(log2 d)
}

void free_group(Group& g) {
  if (g.gexec) cudaGraphExecDestroy(g.gexec);
  g.gexec = nullptr;
}

inline size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" bk_status bk_solve_batched(bk_ctx* c, int32_t n, const bk_operator* A, const double* mu,
                                      const double* const* b, double* const* x, const bk_opts* opts_in,
                                      bk_info* infos) {
  if (!c || n < 1 || !A || !mu || !b || !x) return BK_ERR_ARG;
  err_ctx() = c;
  c->last_error[0] = 0;
  bk_opts opts;
  if (opts_in)
    opts = *opts_in;
  else
    bk_default_opts(&opts);
  if (!(opts.tol > 0.0) || opts.max_loads < 1 || opts.max_refine < 1 || opts.check_every < 1 ||
      !(opts.inner_tol > 0.0) || opts.timeout_cycles < 0)
    return BK_ERR_ARG;
  if (opts.inner != BK_PREC_FP64 && opts.inner != BK_PREC_FP32) return BK_ERR_UNSUPPORTED;
  const int is64 = opts.inner == BK_PREC_FP64;
  const int vals_f64 = A[0].dtype == BK_F64;
  for (int i = 0; i < n; ++i) {
    const bk_operator& o = A[i];
    if (o.kind != BK_DENSE) return BK_ERR_UNSUPPORTED;
    if (o.dtype != A[0].dtype) return BK_ERR_ARG;
    if (!o.vals || o.rows <= 0 || o.rows != o.cols || o.ld < o.cols || !b[i] || !x[i]) return BK_ERR_ARG;
    if (!(mu[i] >= 0.0) || !std::isfinite(mu[i])) return BK_ERR_ARG;
  }
  if (!is64 && vals_f64) return BK_ERR_UNSUPPORTED;  // FP32 blocks take FP32 values
  BK_CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  cudaEvent_t ev0, ev1;
  BK_CK(cudaEventCreate(&ev0));
  BK_CK(cudaEventCreate(&ev1));
  BK_CK(cudaEventRecord(ev0, st));
  if (infos) std::memset(infos, 0, sizeof(bk_info) * n);

  // block width per system: fixed sketch, or the autotune table (nearest size bucket)
  // and the block-product kernel per system (kernel codes: 1 tensor cores where usable,
  // 0 CUDA cores with 16-row tiles, 2 CUDA cores with 32-row tiles)
  std::vector<int> ms(n), want_tc(n, 1);
  for (int i = 0; i < n; ++i) {
    int l = opts.sketch;
    if (l < 0) {
      l = 16;  // untuned default
      int bkt = size_bucket(A[i].rows), bestd = 1 << 30;
      for (auto& kv : c->tune)
        if (std::abs(kv.first - bkt) < bestd) {
          bestd = std::abs(kv.first - bkt);
          l = kv.second;
          auto it = c->tune_tc.find(kv.first);
          want_tc[i] = it == c->tune_tc.end() ? 1 : it->second;
        }
    }
    if (c->force_tc >= 0) want_tc[i] = c->force_tc;
    ms[i] = (int)std::min<int64_t>((int64_t)l + 1, A[i].rows);
    if (bk::padded_width(ms[i]) < 0) return BK_ERR_UNSUPPORTED;
  }
  // groups by padded width and product kernel (key 4 mp + kernel code)
  std::map<int, Group> groups;
  for (int i = 0; i < n; ++i) groups[4 * bk::padded_width(ms[i]) + want_tc[i]].members.push_back(i);

  const size_t es = is64 ? 8 : 4;
  const size_t vs = vals_f64 ? 8 : 4;
  const double rank_tol = is64 ? 1e-12 : 1e-6;
  const int sms = c->sms > 0 ? c->sms : 152;
  std::vector<double> bnorm(n, 0.0), rnorm(n, 0.0);
  std::vector<int> loads(n, 0), refine(n, 0), status(n, BK_NOT_CONVERGED), defl(n, 0);
  // per-system inner target floor and the target and residual of the last pass (the
  // rule of bk_solve: after a pass that met its target but reduced the FP64 residual by
  // far less, later passes stop at half the reduction it achieved)
  std::vector<double> floor_t(n, 0.0), last_t(n, 0.0), last_r(n, 0.0);
  // systems that stopped: a pass that lost its recurrence (BK_BREAKDOWN: residual not
  // finite, or a breakdown that did not reduce it; the next pass would repeat it) or two
  // passes that reduced the residual less than twofold (BK_STAGNATED), and the count of
  // such slow passes
  std::vector<int> failed(n, 0), stag(n, 0);
  bk_status result = BK_OK;
  std::vector<Group*> glist;
  auto cleanup = [&]() {
    for (auto& kv : groups) free_group(kv.second);
  };
#define BK_CKG(expr)                                                              \
  do {                                                                            \
    cudaError_t e_ = (expr);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      bk_status s_ = bkx::from_cuda(e_, #expr, __LINE__, __FILE__);               \
      cleanup();                                                                  \
      return s_;                                                                  \
    }                                                                             \
  } while (0)
  // layout pass: descriptors, thread-block ranges and arena offsets
  size_t arena = up256(sizeof(bk::DevState) * n), vals_bytes = 0;
  int total_cta = 0;
  for (auto& kv : groups) {
    Group& g = kv.second;
    g.mp = kv.first / 4;
    glist.push_back(&g);
    g.tile_rows = (kv.first & 3) == 2 ? 32 : 16;
    // the tensor-core product needs FP32 values with 16-byte aligned rows (host values
    // are staged to 256-byte aligned buffers with the caller's lda)
    g.tc = !is64 && (kv.first & 3) == 1;
    for (int i : g.members) {
      const bool dev = bkx::is_device_ptr(A[i].vals);
      const void* probe = dev ? A[i].vals : reinterpret_cast<const void*>(uintptr_t(256));
      g.tc = g.tc && bk::dense_tc_usable(A[i].rows, probe, A[i].ld, g.mp);
    }
    // thread blocks per system: proportional to d^2 m, at least one, at most its row tiles
    double wsum = 0.0;
    for (int i : g.members) wsum += (double)A[i].rows * A[i].rows * ms[i];
    const int budget = sms * 6;
    for (size_t k = 0; k < g.members.size(); ++k) {
      const int i = g.members[k];
      const int64_t d = A[i].rows;
      const int64_t tiles = (d + 127) / 128;
      int nc = (int)std::lround(budget * (double)d * d * ms[i] / wsum);
      nc = (int)std::max<int64_t>(1, std::min<int64_t>(nc, tiles));
      bk::BSys s;
      std::memset(&s, 0, sizeof(s));
      s.d = d;
      s.lda = A[i].ld;
      s.ld = (d + 31) & ~int64_t(31);
      s.m = ms[i];
      s.cta0 = g.ncta;
      s.ncta = nc;
      s.index = i;
      s.mu = mu[i];
      for (int q = 0; q < nc; ++q) g.hcta.push_back((int)k);
      g.ncta += nc;
      if (!bkx::is_device_ptr(A[i].vals)) vals_bytes += up256(((size_t)(d - 1) * A[i].ld + d) * vs);
      // every block holds all mp / 4 panels of the padded width: the block kernels are
      // compiled for that width and read or write the padding panels as zeros
      const size_t blk = up256((size_t)s.ld * g.mp * es);
      const int ne = bk::gram_entries(g.mp);
      const int rtiles = bk::dense_tc_tiles(d);
      s.npG = g.tc ? rtiles : nc;
      arena += 3 * blk + 4 * up256((size_t)d * 8) + up256((size_t)ne * s.npG * 8) + up256((size_t)ne * nc * 8) +
               up256((size_t)s.m * 8) + 3 * up256((size_t)g.mp * g.mp * es) + up256((size_t)g.mp * es);
      if (g.tc) {
        arena += up256(bk::dense_tc_pt_bytes(d, g.mp));
        for (int t = 0; t < rtiles; ++t) g.htile.push_back((int)k);
      }
      g.hs.push_back(s);
    }
    if (g.tc) {
      const size_t nt = g.htile.size();
      g.htile.resize(2 * nt);
      size_t t = 0;
      for (size_t k = 0; k < g.hs.size(); ++k)
        for (int r = 0; r < bk::dense_tc_tiles(g.hs[k].d); ++r) g.htile[nt + t++] = r;
      g.btc.ntiles = (int)nt;
      arena += up256(sizeof(int) * 2 * nt) + up256(sizeof(CUtensorMap) * 2 * g.hs.size());
    }
    arena += up256(sizeof(bk::BSys) * g.hs.size()) + up256(sizeof(int) * g.hcta.size());
    total_cta = std::max(total_cta, g.ncta);
  }
  arena += up256(sizeof(double) * (total_cta + 16));
  char* base = nullptr;
  char* vbase = nullptr;
  BK_CKG(ws_get(c, WS_BATCH, arena, (void**)&base));
  if (vals_bytes) BK_CKG(ws_get(c, WS_BATCH_VALS, vals_bytes, (void**)&vbase));
  char* q = base;
  auto take = [&](size_t nb) {
    char* r = q;
    q += up256(nb);
    return (void*)r;
  };
  bk::DevState* dstates = (bk::DevState*)take(sizeof(bk::DevState) * n);
  double* rparts = (double*)take(sizeof(double) * (total_cta + 16));
  for (Group* g : glist) {
    g->ds = (bk::BSys*)take(sizeof(bk::BSys) * g->hs.size());
    g->cta_sys = (int*)take(sizeof(int) * g->hcta.size());
    BK_CKG(cudaMemcpyAsync(g->cta_sys, g->hcta.data(), sizeof(int) * g->hcta.size(), cudaMemcpyHostToDevice, st));
    for (bk::BSys& s : g->hs) {
      const int i = s.index;
      const int64_t d = s.d;
      s.st = dstates + i;
      if (bkx::is_device_ptr(A[i].vals)) {
        s.A = A[i].vals;
      } else {
        const size_t vb = ((size_t)(d - 1) * A[i].ld + d) * vs;
        BK_CKG(cudaMemcpyAsync(vbase, A[i].vals, vb, cudaMemcpyHostToDevice, st));
        s.A = vbase;
        vbase += up256(vb);
      }
      s.A64 = s.A;
      const size_t blk = (size_t)s.ld * g->mp * es;
      const int ne = bk::gram_entries(g->mp);
      s.P = take(blk);
      s.Q = take(blk);
      s.Y = take(blk);
      BK_CKG(cudaMemsetAsync(s.P, 0, 3 * up256(blk), st));  // padding columns stay zero
      s.xin = (double*)take((size_t)d * 8);
      s.x64 = (double*)take((size_t)d * 8);
      s.r64 = (double*)take((size_t)d * 8);
      double* bcopy = (double*)take((size_t)d * 8);
      s.Gp = (double*)take((size_t)ne * s.npG * 8);
      s.Sp = (double*)take((size_t)ne * s.ncta * 8);
      s.cvec = (double*)take((size_t)s.m * 8);
      s.gi_t = take((size_t)g->mp * g->mp * es);
      s.ti_t = take((size_t)g->mp * g->mp * es);
      s.t_t = take((size_t)g->mp * g->mp * es);
      s.xc_t = take((size_t)g->mp * es);
      s.pt = nullptr;
      if (g->tc) s.pt = (float*)take(bk::dense_tc_pt_bytes(d, g->mp));
      BK_CKG(cudaMemcpyAsync(bcopy, b[i], (size_t)d * 8, cudaMemcpyDefault, st));
      s.b = bcopy;
      BK_CKG(cudaMemsetAsync(s.x64, 0, (size_t)d * 8, st));
    }
  }
  // tensor-core groups: tile tables and the two tensor maps of every system
  for (Group* g : glist) {
    if (!g->tc) continue;
    int* tiles = (int*)take(sizeof(int) * g->htile.size());
    CUtensorMap* maps = (CUtensorMap*)take(sizeof(CUtensorMap) * 2 * g->hs.size());
    g->hmaps.resize(2 * g->hs.size());
    for (size_t k = 0; k < g->hs.size(); ++k) {
      const bk::BSys& s = g->hs[k];
      BK_CKG(bk::tc_make_maps(g->mp, s.d, (const float*)s.A, s.lda, s.pt, &g->hmaps[2 * k]));
    }
    BK_CKG(cudaMemcpyAsync(tiles, g->htile.data(), sizeof(int) * g->htile.size(), cudaMemcpyHostToDevice, st));
    BK_CKG(cudaMemcpyAsync(maps, g->hmaps.data(), sizeof(CUtensorMap) * g->hmaps.size(), cudaMemcpyHostToDevice, st));
    g->btc.tile_sys = tiles;
    g->btc.tile_row = tiles + g->btc.ntiles;
    g->btc.maps = maps;
    g->btc.wait_cycles = opts.timeout_cycles;
  }
  std::vector<double> hparts(total_cta + 16);
  std::vector<bk::DevState> hst(n);

  // FP64 residual of every system (x64 as it stands) -> rnorm
  auto residuals = [&]() -> cudaError_t {
    for (Group* g : glist) {
      cudaError_t e = cudaMemcpyAsync(g->ds, g->hs.data(), sizeof(bk::BSys) * g->hs.size(),
                                      cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return e;
      if ((e = bk::launch_batch_resid(vals_f64, g->ds, g->cta_sys, g->ncta, rparts, st)) != cudaSuccess) return e;
      if ((e = cudaMemcpyAsync(hparts.data(), rparts, sizeof(double) * g->ncta, cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess)
        return e;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
      for (size_t k = 0; k < g->hs.size(); ++k) {
        const bk::BSys& s = g->hs[k];
        double ss = 0.0;
        for (int q = 0; q < s.ncta; ++q) ss += hparts[s.cta0 + q];
        rnorm[s.index] = std::sqrt(ss);
      }
    }
    return cudaSuccess;
  };
  BK_CKG(residuals());
  for (int i = 0; i < n; ++i) bnorm[i] = rnorm[i];

  const bool use_graph = std::getenv("BK_NO_GRAPH") == nullptr;
  for (int pass = 0; pass < opts.max_refine; ++pass) {
    int nactive = 0;
    for (Group* g : glist) {
      for (bk::BSys& s : g->hs) {
        const int i = s.index;
        const bool conv = rnorm[i] <= opts.tol * bnorm[i];
        if (conv) status[i] = BK_OK;
        s.active = (!conv && loads[i] < opts.max_loads && !failed[i]) ? 1 : 0;
        nactive += s.active;
        s.rnorm = rnorm[i];
        s.rscale = rnorm[i] > 0 ? 1.0 / rnorm[i] : 0.0;
        double target = std::max(std::max(opts.inner_tol, 0.5 * opts.tol * bnorm[i] / std::max(rnorm[i], 1e-300)),
                                 floor_t[i]);
        s.tol_abs = std::min(target, 0.5);
        last_t[i] = s.tol_abs;
        last_r[i] = rnorm[i];
        s.max_loads = std::max(1, opts.max_loads - loads[i]);
      }
    }
    if (nactive == 0) break;
    for (Group* g : glist) {
      BK_CKG(cudaMemcpyAsync(g->ds, g->hs.data(), sizeof(bk::BSys) * g->hs.size(), cudaMemcpyHostToDevice, st));
      BK_CKG(bk::launch_batch_start(is64, g->mp, g->ds, (int)g->hs.size(), g->cta_sys, g->ncta, opts.seed, rank_tol,
                                    st));
    }
    // inner solves of all groups, chunks of check_every steps
    for (int chunk = 0;; ++chunk) {
      for (Group* g : glist) {
        if (use_graph && chunk > 0) {
          if (!g->gexec) {
            cudaGraph_t graph;
            BK_CKG(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
            cudaError_t ce = cudaSuccess;
            for (int it = 0; it < opts.check_every && ce == cudaSuccess; ++it)
              ce = bk::launch_batch_step(is64, vals_f64, g->mp, g->ds, (int)g->hs.size(), g->cta_sys, g->ncta,
                                         rank_tol, g->tc ? &g->btc : nullptr, g->tile_rows, st);
            cudaError_t ee = cudaStreamEndCapture(st, &graph);
            BK_CKG(ce);
            BK_CKG(ee);
            ee = cudaGraphInstantiate(&g->gexec, graph, 0);
            cudaGraphDestroy(graph);
            BK_CKG(ee);
          }
          BK_CKG(cudaGraphLaunch(g->gexec, st));
        } else {
          for (int it = 0; it < opts.check_every; ++it)
            BK_CKG(bk::launch_batch_step(is64, vals_f64, g->mp, g->ds, (int)g->hs.size(), g->cta_sys, g->ncta,
                                         rank_tol, g->tc ? &g->btc : nullptr, g->tile_rows, st));
        }
      }
      BK_CKG(cudaMemcpyAsync(hst.data(), dstates, sizeof(bk::DevState) * n, cudaMemcpyDeviceToHost, st));
      BK_CKG(cudaStreamSynchronize(st));
      // a tensor-core product whose pipeline wait gave up left an invalid block: stop
      bool timed_out = false;
      for (int i = 0; i < n; ++i) timed_out = timed_out || hst[i].timeout != 0;
      if (timed_out) {
        std::snprintf(c->last_error, sizeof(c->last_error), "tensor-core pipeline wait timed out");
        for (int i = 0; i < n; ++i)
          if (infos) {
            infos[i].status = BK_TIMEOUT;
            infos[i].loads = loads[i] + hst[i].loads;
            infos[i].refinements = refine[i];
          }
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        cleanup();
        return BK_TIMEOUT;
      }
      bool all = true;
      for (int i = 0; i < n; ++i) all = all && (hst[i].done_a || hst[i].done_b);
      if (all) break;
    }
    for (Group* g : glist)
      for (bk::BSys& s : g->hs)
        if (s.active) {
          loads[s.index] += hst[s.index].loads;
          refine[s.index] += 1;
          defl[s.index] += s.m - hst[s.index].kept;
        }
    std::vector<int> conv_inner(n, 0);
    for (int i = 0; i < n; ++i) conv_inner[i] = hst[i].status == bk::ST_CONVERGED;
    for (Group* g : glist) {
      BK_CKG(cudaMemcpyAsync(g->ds, g->hs.data(), sizeof(bk::BSys) * g->hs.size(), cudaMemcpyHostToDevice, st));
      BK_CKG(bk::launch_batch_axpy(g->ds, g->cta_sys, g->ncta, st));
    }
    BK_CKG(residuals());
    bool any_revert = false;
    for (Group* g : glist)
      for (bk::BSys& s : g->hs) {
        const int i = s.index;
        const bool ran = s.active && last_r[i] > 0.0;
        s.active = 0;
        if (!ran) continue;
        // a residual that is not finite, or a breakdown that did not reduce it: the pass
        // lost its recurrence (the rule of bk_solve)
        if (!std::isfinite(rnorm[i]) || (hst[i].status == bk::ST_BREAKDOWN && !(rnorm[i] < last_r[i]))) {
          failed[i] = BK_BREAKDOWN;
          if (is64) {  // undo x += ||r|| xin (FP32 systems are solved again below)
            s.active = 1;
            s.rnorm = -s.rnorm;
            any_revert = true;
          }
          continue;
        }
        const double achieved = rnorm[i] / last_r[i];
        if (conv_inner[i] && achieved > 4.0 * last_t[i]) floor_t[i] = 0.5 * achieved;
        if (!(achieved < 0.5) && ++stag[i] >= 2) failed[i] = BK_STAGNATED;
      }
    if (any_revert) {
      for (Group* g : glist) {
        BK_CKG(cudaMemcpyAsync(g->ds, g->hs.data(), sizeof(bk::BSys) * g->hs.size(), cudaMemcpyHostToDevice, st));
        BK_CKG(bk::launch_batch_axpy(g->ds, g->cta_sys, g->ncta, st));
      }
      BK_CKG(residuals());
    }
  }
  for (int i = 0; i < n; ++i) {
    if (rnorm[i] <= opts.tol * bnorm[i])
      status[i] = BK_OK;
    else if (failed[i])
      status[i] = failed[i];
    if (status[i] != BK_OK) result = BK_NOT_CONVERGED;
  }
  for (Group* g : glist)
    for (bk::BSys& s : g->hs) BK_CKG(cudaMemcpyAsync(x[s.index], s.x64, (size_t)s.d * 8, cudaMemcpyDefault, st));
  BK_CKG(cudaEventRecord(ev1, st));
  BK_CKG(cudaEventSynchronize(ev1));
  float ms_total = 0.f;
  cudaEventElapsedTime(&ms_total, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (infos)
    for (int i = 0; i < n; ++i) {
      infos[i].status = status[i];
      infos[i].loads = loads[i];
      infos[i].refinements = refine[i];
      infos[i].residual_loads = refine[i] + 1;
      infos[i].rel_residual = bnorm[i] > 0 ? rnorm[i] / bnorm[i] : 0.0;
      infos[i].ms_total = ms_total;
      infos[i].deflations = defl[i];
    }
  cleanup();
#undef BK_CKG
  if (is64) return result;
  // FP32 blocks stopped reducing these systems' residuals: they are solved again from
  // x = 0 in FP64 blocks (the FP32 values promoted in the products), in one nested batch
  std::vector<int> redo;
  int max_used = 0;
  for (int i = 0; i < n; ++i)
    if (failed[i] && status[i] != BK_OK) {
      redo.push_back(i);
      max_used = std::max(max_used, loads[i]);
    }
  if (redo.empty() || max_used >= opts.max_loads) return result;
  const int nr = (int)redo.size();
  std::vector<bk_operator> ra((size_t)nr);
  std::vector<double> rmu((size_t)nr);
  std::vector<const double*> rb((size_t)nr);
  std::vector<double*> rx((size_t)nr);
  std::vector<bk_info> ri((size_t)nr);
  for (int k = 0; k < nr; ++k) {
    ra[k] = A[redo[k]];
    rmu[k] = mu[redo[k]];
    rb[k] = b[redo[k]];
    rx[k] = x[redo[k]];
  }
  bk_opts o64 = opts;
  o64.inner = BK_PREC_FP64;
  o64.max_loads = opts.max_loads - max_used;
  const bk_status rs = bk_solve_batched(c, nr, ra.data(), rmu.data(), rb.data(), rx.data(), &o64, ri.data());
  if (rs != BK_OK && rs != BK_NOT_CONVERGED) return rs;
  result = BK_OK;
  for (int k = 0; k < nr; ++k) status[redo[k]] = ri[k].status;
  for (int i = 0; i < n; ++i)
    if (status[i] != BK_OK) result = BK_NOT_CONVERGED;
  if (infos) {
    for (int k = 0; k < nr; ++k) {
      bk_info& f = infos[redo[k]];
      f.status = ri[k].status;
      f.loads += ri[k].loads;
      f.refinements += ri[k].refinements;
      f.residual_loads += ri[k].residual_loads;
      f.rel_residual = ri[k].rel_residual;
      f.deflations += ri[k].deflations;
      f.fp64_fallback = 1;
    }
    for (int i = 0; i < n; ++i) infos[i].ms_total += ri[0].ms_total;
  }
  return result;
}

extern "C" bk_status bk_autotune(bk_ctx* c, int32_t n, const bk_operator* A, const double* mu,
                                 const double* const* b, const int32_t* candidates, int32_t ncand,
                                 const bk_opts* opts_in, int32_t* chosen) {
  if (!c || n < 1 || !A || !mu || !b || !candidates || ncand < 1) return BK_ERR_ARG;
  bk_opts opts;
  if (opts_in)
    opts = *opts_in;
  else
    bk_default_opts(&opts);
  // Per size bucket, the bucket's calibration systems are solved together as one batch,
  // repeated until the batch streams at least kBatchBytes of matrix per load (up to
  // kMaxCopies copies, each with its own x), so that the timing reflects the systems'
  // cost inside a large batch rather than the per-step latency of a tiny one. Each
  // candidate is timed three times after a warm solve (best of three); a candidate
  // that leaves any system unconverged is out for the bucket.
  constexpr double kBatchBytes = 1e9;
  constexpr int kMaxCopies = 64;
  std::map<int, std::vector<int>> buckets;
  for (int i = 0; i < n; ++i) {
    if (A[i].rows < 1) return BK_ERR_ARG;
    buckets[size_bucket(A[i].rows)].push_back(i);
  }
  for (int k = 0; k < ncand; ++k)
    if (candidates[k] < 1) return BK_ERR_ARG;
  for (auto& kv : buckets) {
    const std::vector<int>& mem = kv.second;
    double bytes = 0.0;
    for (int i : mem) bytes += (double)A[i].rows * A[i].rows * (A[i].dtype == BK_F64 ? 8 : 4);
    const int copies = (int)std::min<double>(kMaxCopies, std::max(1.0, std::ceil(kBatchBytes / bytes)));
    std::vector<bk_operator> ops;
    std::vector<double> mus;
    std::vector<const double*> bs;
    std::vector<std::vector<double>> xs;
    for (int r = 0; r < copies; ++r)
      for (int i : mem) {
        ops.push_back(A[i]);
        mus.push_back(mu[i]);
        bs.push_back(b[i]);
        xs.emplace_back((size_t)A[i].rows, 0.0);
      }
    std::vector<double*> xp(xs.size());
    for (size_t q = 0; q < xs.size(); ++q) xp[q] = xs[q].data();
    const int nb = (int)ops.size();
    std::vector<bk_info> infos((size_t)nb);
    double best_t = INFINITY;
    int best_k = -1;
    for (int k = 0; k < ncand; ++k) {
      bk_opts o = opts;
      o.sketch = candidates[k];
      double t = INFINITY;
      for (int rep = 0; rep < 4; ++rep) {  // a warm solve, then three timed ones
        bk_status s = bk_solve_batched(c, nb, ops.data(), mus.data(), bs.data(), xp.data(), &o, infos.data());
        if (s == BK_ERR_UNSUPPORTED) {  // a block width the kernels are not built for
          t = INFINITY;
          break;
        }
        if (s != BK_OK && s != BK_NOT_CONVERGED) return s;
        if (s != BK_OK) {
          t = INFINITY;
          break;
        }
        if (rep > 0) t = std::min(t, (double)infos[0].ms_total);
      }
      if (t < best_t) {
        best_t = t;
        best_k = k;
      }
    }
    if (best_k < 0) continue;
    c->tune[kv.first] = candidates[best_k];
    // product kernel and tile shape of the winning width: the default (tensor cores for
    // FP32 blocks where the width is one they are built for, else 16-row FFMA tiles)
    // against the other kernels, timed the same way
    const bool tc_built = opts.inner == BK_PREC_FP32 && bk::padded_width(candidates[best_k] + 1) <= bk::kTcMaxPadded;
    const int def = tc_built ? 1 : 0;
    c->tune_tc[kv.first] = def;
    for (int kern : {0, 1, 2}) {
      if (kern == def || (kern == 1 && !tc_built)) continue;
      bk_opts o = opts;
      o.sketch = candidates[best_k];
      double t = INFINITY;
      c->force_tc = kern;
      for (int rep = 0; rep < 4; ++rep) {
        bk_status s = bk_solve_batched(c, nb, ops.data(), mus.data(), bs.data(), xp.data(), &o, infos.data());
        if (s != BK_OK) {
          t = INFINITY;
          if (s != BK_NOT_CONVERGED) {
            c->force_tc = -1;
            return s;
          }
          break;
        }
        if (rep > 0) t = std::min(t, (double)infos[0].ms_total);
      }
      c->force_tc = -1;
      if (t < best_t) {
        best_t = t;
        c->tune_tc[kv.first] = kern;
      }
    }
  }
  if (chosen)
    for (int i = 0; i < n; ++i) {
      auto it = c->tune.find(size_bucket(A[i].rows));
      chosen[i] = it == c->tune.end() ? -1 : it->second;
    }
  return BK_OK;
}

extern "C" bk_status bk_autotune_save(const bk_ctx* c, const char* path) {
  if (!c || !path) return BK_ERR_ARG;
  FILE* f = std::fopen(path, "w");
  if (!f) return BK_ERR_ARG;
  std::fprintf(f, "# bk autotune table: floor(log2 d) sketch product(1 tensor-core, 0 cuda-core 16-row tiles, "
                 "2 cuda-core 32-row tiles)\n");
  for (auto& kv : c->tune) {
    auto it = c->tune_tc.find(kv.first);
    std::fprintf(f, "%d %d %d\n", kv.first, kv.second, it == c->tune_tc.end() ? 1 : it->second);
  }
  const bool ok = std::fclose(f) == 0;
  return ok ? BK_OK : BK_ERR_ARG;
}

extern "C" bk_status bk_autotune_load(bk_ctx* c, const char* path) {
  if (!c || !path) return BK_ERR_ARG;
  FILE* f = std::fopen(path, "r");
  if (!f) return BK_ERR_ARG;
  std::map<int, int> tune, tune_tc;
  char line[256];
  bk_status st = BK_OK;
  while (std::fgets(line, sizeof(line), f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    int bkt = 0, sk = 0, tc = 1;
    if (std::sscanf(line, "%d %d %d", &bkt, &sk, &tc) != 3 || bkt < 0 || bkt > 62 || sk < 1 || tc < 0 || tc > 2) {
      st = BK_ERR_ARG;
      break;
    }
    tune[bkt] = sk;
    tune_tc[bkt] = tc;
  }
  std::fclose(f);
  if (st != BK_OK) return st;
  c->tune = tune;
  c->tune_tc = tune_tc;
  return BK_OK;
}
