// dataset_launch.cuh -- the adaptive rounds over a resident dataset for one
// element type of the gathered copy: round-0 pass (per-pair draws over staged
// rows, or the shared-coordinate pass), then the round-loop kernel, query
// chunk by query chunk. Instantiated for the nine element types across
// several translation units (ds_launch_*.cu) so they compile in parallel.
#pragma once

#include "adaptive_kernel.cuh"

namespace knn {

// Per-query k and counter ids of a mixed batch (null: one k, ids qid_base + q).
struct MixedBatch {
  const int32_t* kq = nullptr;
  const uint64_t* qids = nullptr;
  int32_t h_per_k = 0;
  int32_t out_stride = 0;
};

template <class E>
knn_status adaptive_ds_launch(const knn_dataset* ds, const float* Q, int32_t nq, int32_t k, double delta,
                                     uint64_t seed, const knn_opts& o, int64_t* out_idx, int32_t* out_count,
                                     int64_t* out_evals, int32_t* out_rounds, int32_t* log_code, float* log_S,
                                     void* workspace, size_t workspace_bytes, cudaStream_t stream,
                                     const MixedBatch* mix = nullptr) {
  const int64_t n = ds->n;
  const int32_t m = ds->m;
  // round 0 point-major: the shared form for B0 <= 64, the staged-rows pass otherwise
  const bool r0 = E::kPerm ? (o.B0 < m && o.B0 <= 64) : round0_applies(m, o);
  AdaptivePlan p;
  knn_status s = plan_adaptive<E>(n, m, nq, k, &o, &p);
  if (s != KNN_OK) return s;
  const int chunk = r0 ? round0_chunk(n, nq, p.grid) : nq;
  // round-0 tile minima: per CTA of the staged-rows pass, per warp of the shared pass
  const int rows = round0_rows(m, o.B0);
  const int tiles = !r0 ? 0 : (int)(E::kPerm ? (n + 31) / 32 : (n + rows - 1) / rows);
  Carve measure;
  carve_adaptive(measure, n, p, nullptr);
  const int qpw = E::kPerm && r0 ? (o.B0 <= 16 ? 16 : (o.B0 <= 32 ? 32 : 64)) : 0;  // staged by round 0
  // round 0 under shared coordinates as a tensor-core contraction (squared l2)
  const bool r0tc = E::kPerm && r0 && o.r0_tensor && o.metric == KNN_METRIC_L2SQ && ds->r0op[E::kStorage];
  if (r0) {
    measure.take<float>((size_t)chunk * (size_t)n);
    measure.take<float>((size_t)chunk * (size_t)tiles);
    measure.take<float>((size_t)chunk * (size_t)qpw);
    if (r0tc) measure.take<uint8_t>(round0_tc_scratch(n, chunk));
  }
  const bool order = o.query_order && chunk >= 2 && chunk <= kOrderMax;
  if (order) measure.take<uint8_t>(query_order_scratch(m, chunk));
  const size_t need = measure.off + 256;
  Workspace ws;
  s = ws.acquire(workspace, workspace_bytes, need, stream);
  if (s != KNN_OK) return s;
  Carve cv;
  cv.base = reinterpret_cast<uint8_t*>(((uintptr_t)ws.ptr + 255) & ~uintptr_t(255));
  AdaptiveCarve c;
  carve_adaptive(cv, n, p, &c);
  float* r0buf = r0 ? cv.take<float>((size_t)chunk * (size_t)n) : nullptr;
  float* r0min = r0 ? cv.take<float>((size_t)chunk * (size_t)tiles) : nullptr;
  float* qperm = qpw ? cv.take<float>((size_t)chunk * (size_t)qpw) : nullptr;
  uint8_t* r0scratch = r0tc ? cv.take<uint8_t>(round0_tc_scratch(n, chunk)) : nullptr;
  uint8_t* oscratch = order ? cv.take<uint8_t>(query_order_scratch(m, chunk)) : nullptr;
  int32_t* qorder = order ? reinterpret_cast<int32_t*>(oscratch + query_order_scratch(m, chunk) -
                                                       ((size_t)chunk * 4 + 255) / 256 * 256)
                          : nullptr;
  AdaptiveArgs a;
  const void* G = ds->X;
  if (E::kStorage == KNN_STORE_BF16) G = ds->xb;
  if (E::kStorage == KNN_STORE_FP8) G = ds->x8;
  if (E::kPerm) G = E::kStorage == KNN_STORE_BF16 ? (const void*)ds->pb
                    : (E::kStorage == KNN_STORE_FP8 ? (const void*)ds->p8 : (const void*)ds->p32);
  a.X = ds->X;
  a.G = G;
  a.gscale = ds->scale8;
  a.emax = E::kStorage == KNN_STORE_F32 ? nullptr : reinterpret_cast<const float*>(ds->emax + E::kStorage);
  a.Q = Q;
  a.n = n;
  a.m = m;
  a.nq = nq;
  a.k = k;
  a.h = o.h;
  a.kq = mix ? mix->kq : nullptr;
  a.qids = mix ? mix->qids : nullptr;
  a.h_per_k = mix ? mix->h_per_k : 0;
  a.out_stride = mix ? mix->out_stride : k + o.h;
  a.bound = o.bound;
  const double dprime = delta / (double)n;
  a.a_c0 = 0.0f;
  a.a_c1 = 0.0f;
  if (o.bound == KNN_BOUND_FOOTNOTE)
    a.a_c0 = (float)(std::log(1.0 / dprime) + 3.0 * std::log(std::log(1.0 / dprime)));
  else if (o.bound == KNN_BOUND_LEMMA)
    a.a_c0 = (float)std::log(125.0 / dprime);
  else
    a.a_c1 = (float)((double)n / delta);
  a.c_alpha = (float)o.c_alpha;
  a.B0 = o.B0;
  a.B = o.B;
  a.grow = o.grow;
  a.seed = seed;
  a.rk = philox_keys(seed);
  a.qid_base = o.qid_base;
  a.mask_p = o.mask_p;
  a.mask_q = o.mask_q;
  a.xrange = ds->range;
  a.ws_ids = c.ids;
  a.ws_S = c.S;
  a.ws_C = c.C;
  a.ws_acc_id = c.acc_id;
  a.ws_acc_d = c.acc_d;
  a.ws_acc_U = c.acc_U;
  a.ws_acc_L = c.acc_L;
  a.acc_cap = p.acc_cap;
  a.ws_F = c.F;
  a.fuse_cap = p.fuse_cap;
  a.queue = c.queue;
  a.out_idx = out_idx;
  a.out_count = out_count;
  a.out_evals = out_evals;
  a.out_rounds = out_rounds;
  a.log_code = log_code;
  a.log_S = log_code ? log_S : nullptr;
  a.vec = (m % 4 == 0) && (((uintptr_t)ds->X & 15) == 0);
  set_blocks<E>(a, o);
  a.R0 = r0buf;
  a.R0min = r0min;
  a.r0tiles = tiles;
  a.jperm = ds->jperm;
  a.mp = ds->mp;
  a.phase_clk = phase_clocks_ptr();
  a.r0_resum = r0tc ? 1 : 0;
  if (r0 && !E::kPerm) {
    s = cuda_check(cudaFuncSetAttribute(a.l1 ? reinterpret_cast<const void*>(round0_kernel<E, true>)
                                             : reinterpret_cast<const void*>(round0_kernel<E, false>),
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)((size_t)rows * m * 4)),
                   "cudaFuncSetAttribute(round0)");
    if (s != KNN_OK) {
      ws.release();
      return s;
    }
  }
  // queries in chunks whose round-0 sums fit the buffer: round 0 point-major,
  // then the remaining rounds of the chunk's queries
  for (int32_t q0 = 0; q0 < nq && s == KNN_OK; q0 += chunk) {
    AdaptiveArgs ac = a;
    ac.nq = std::min(chunk, nq - q0);
    ac.Q = Q + (size_t)q0 * m;
    ac.out_idx = out_idx + (size_t)q0 * a.out_stride;
    ac.out_count = out_count + q0;
    ac.out_evals = out_evals + q0;
    ac.out_rounds = out_rounds ? out_rounds + q0 : nullptr;
    ac.log_code = log_code ? log_code + (size_t)q0 * n : nullptr;
    ac.log_S = a.log_S ? a.log_S + (size_t)q0 * n : nullptr;
    ac.kq = a.kq ? a.kq + q0 : nullptr;
    ac.qids = a.qids ? a.qids + q0 : nullptr;
    ac.qid_base = a.qid_base + (uint64_t)q0;
    s = cuda_check(cudaMemsetAsync(c.queue, 0, 4, stream), "memset(queue)");
    if (s == KNN_OK && order && ac.nq >= 2) {  // the chunk's locality order (before the round-0 pass)
      s = launch_query_order(ac.Q, ac.nq, m, oscratch, qorder, stream);
      ac.qorder = qorder;
    }
    if (r0) kernel_mark(stream, 0);
    if (s == KNN_OK && r0tc) {
      s = round0_tc(ds, E::kStorage, ac.Q, ac.nq, o.B0, r0buf, r0min, tiles, r0scratch, stream);
    } else if (s == KNN_OK && r0) {
      if constexpr (E::kPerm) {
        const unsigned blocks = (unsigned)((n + kR0SharedThreads - 1) / kR0SharedThreads);
        const int64_t cnt = (int64_t)ac.nq * qpw;
        permute_query_columns_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, stream>>>(ac.Q, m, ac.nq, ds->jperm,
                                                                                         o.B0, qpw, qperm);
        s = cuda_check(cudaGetLastError(), "permute_query_columns_kernel launch");
        if (s != KNN_OK) break;
        if (o.B0 <= 16) {
          const dim3 grid(blocks, (unsigned)((ac.nq + R0SharedCfg<2>::kQueries - 1) / R0SharedCfg<2>::kQueries));
          (a.l1 ? round0_shared_kernel<E, 2, true> : round0_shared_kernel<E, 2, false>)
              <<<grid, kR0SharedThreads, 0, stream>>>(ac, qperm, r0buf, r0min);
        } else if (o.B0 <= 32) {
          const dim3 grid(blocks, (unsigned)((ac.nq + R0SharedCfg<4>::kQueries - 1) / R0SharedCfg<4>::kQueries));
          (a.l1 ? round0_shared_kernel<E, 4, true> : round0_shared_kernel<E, 4, false>)
              <<<grid, kR0SharedThreads, 0, stream>>>(ac, qperm, r0buf, r0min);
        } else {
          const dim3 grid(blocks, (unsigned)((ac.nq + R0SharedCfg<8>::kQueries - 1) / R0SharedCfg<8>::kQueries));
          (a.l1 ? round0_shared_kernel<E, 8, true> : round0_shared_kernel<E, 8, false>)
              <<<grid, kR0SharedThreads, 0, stream>>>(ac, qperm, r0buf, r0min);
        }
        s = cuda_check(cudaGetLastError(), "round0_shared_kernel launch");
      } else {
        const unsigned blocks = (unsigned)((n + rows - 1) / rows);
        (a.l1 ? round0_kernel<E, true> : round0_kernel<E, false>)
            <<<blocks, kR0Threads, (size_t)rows * m * 4, stream>>>(ac, rows, r0buf, r0min);
        s = cuda_check(cudaGetLastError(), "round0_kernel launch");
      }
    }
    kernel_mark(stream, 1);
    if (s == KNN_OK) s = launch_rounds<E>(p, ac, stream);
    kernel_mark(stream, 2);
  }
  ws.release();
  return s;
}


#define KNN_DS_LAUNCH_DECL(E)                                                                                  \
  knn_status adaptive_ds_launch<E>(const knn_dataset*, const float*, int32_t, int32_t, double, uint64_t,         \
                                   const knn_opts&, int64_t*, int32_t*, int64_t*, int32_t*, int32_t*, float*,    \
                                   void*, size_t, cudaStream_t, const MixedBatch*)

}  // namespace knn
