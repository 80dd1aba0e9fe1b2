// Likelihood weighting (§3.6.2) on many independent line-fitting data sets of
// uneven size in one persistent launch.
//
// Work items are (instance, particle tile) pairs.  The host plan orders them
// heaviest first (by data length, the per-trace cost) so the persistent blocks,
// which take items from an atomic queue, end together (longest-processing-time
// order).  Each item reduces its traces to per-degree partials; the last item of
// an instance to finish merges that instance's partials into its summary.  The
// launch itself only clears counters and starts one kernel, so it can be
// captured in a CUDA graph and replayed.  The autotuner picks the traces per
// thread and the resident blocks per SM by timing the candidates, and caches
// the choice in a JSON file.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <numeric>
#include <string>
#include <vector>

#include "kernels.h"
#include "learned.cuh"
#include "posterior.cuh"
#include "trace.cuh"

namespace ppl {

struct BatchItem {
  int32_t inst;
  int32_t tile;
};

// Workspace layout of a prepared plan (offsets from the workspace base).
struct BatchLayout {
  size_t header, items, first, count_tmpl, count, inst_max, parts, total;
};

static size_t align256(size_t v) { return (v + 255) / 256 * 256; }

constexpr int kWarpParts = (kTpb / 32) * kMaxDegrees;  // partials one tile leaves

static BatchLayout batch_layout(int64_t n_items, int32_t n_inst) {
  BatchLayout l;
  size_t off = 0;
  l.header = off;
  off += 512;
  l.items = off;
  off += align256((size_t)n_items * sizeof(BatchItem));
  l.first = off;
  off += align256((size_t)n_inst * sizeof(int32_t));
  l.count_tmpl = off;
  off += align256((size_t)n_inst * sizeof(int32_t));
  l.count = off;
  off += align256((size_t)n_inst * sizeof(int32_t));
  l.inst_max = off;
  off += align256((size_t)n_inst * kMaxDegrees * sizeof(int32_t));
  l.parts = off;
  off += align256((size_t)n_items * kWarpParts * sizeof(DegPartial));
  l.total = off;
  return l;
}

constexpr int kBatchChunk = 4096;  // data points staged in shared memory at a time

template <int PPT, bool LEARNED>
__global__ void __launch_bounds__(kTpb, PPT >= 8 ? 2 : (LEARNED ? 3 : 4)) batched_kernel(
    PolyParams p, const float* __restrict__ xs, const float* __restrict__ ys,
    const int64_t* __restrict__ data_off, const int64_t* __restrict__ part_off,
    const BatchItem* __restrict__ items, int64_t n_items, const int32_t* __restrict__ first,
    int32_t* count, uint64_t seed, const float* __restrict__ proposal, unsigned* inst_max,
    WsHeader* hdr, DegPartial* parts, ppl_is_result* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  TraceSmem<PPT>& ts = *reinterpret_cast<TraceSmem<PPT>*>(smem);
  float2* sdata = reinterpret_cast<float2*>(smem + trace_smem_bytes<PPT>());
  __shared__ DegPartial gout[kMaxDegrees], fin[kMaxDegrees];
  __shared__ float2 fS[kMaxDegrees], fS2[kMaxDegrees];
  __shared__ int64_t item_sh;
  __shared__ bool last_sh;
  __shared__ ProposalSmem prop;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  reset_warp_partials(ts);
  int cur = -1;      // instance whose data is staged
  int cur_prop = -1;  // instance whose proposal is loaded
  while (true) {
    if (tid == 0) item_sh = (int64_t)atomicAdd(&hdr->tile_counter[1], 1u);
    __syncthreads();
    const int64_t it = item_sh;
    if (it >= n_items) break;
    const int b = items[it].inst;
    const int64_t d0 = data_off[b], L = data_off[b + 1] - d0;
    const int64_t N = part_off[b + 1] - part_off[b];
    const bool resident = L <= kBatchChunk;
    if (resident && b != cur) {
      for (int l = tid; l < L; l += kTpb) sdata[l] = make_float2(xs[d0 + l], ys[d0 + l]);
      __syncthreads();
      cur = b;
    } else if (!resident) {
      cur = -1;  // the chunks overwrite the staged data
    }
    const int64_t tbase = (int64_t)items[it].tile * kTpb * PPT;
    // maxima already reached by this instance's finished items bound the final
    // maxima from below: traces far beneath them are skipped (trace_group)
    if (tid < kMaxDegrees) {
      const unsigned k = (unsigned)ld_volatile_i32(reinterpret_cast<const int32_t*>(inst_max) +
                                                   (int64_t)b * kMaxDegrees + tid);
      ts.ext_max[tid] = (k == 0) ? -INFINITY : key_float(k);
    }
    __syncthreads();
    if (LEARNED) {
      if (b != cur_prop) {
        __syncthreads();
        if (tid == 0) load_proposal(p, proposal + (int64_t)b * 48, prop);
        __syncthreads();
        cur_prop = b;
      }
      trace_group<PPT>(LearnedDraw{p, seed, (uint32_t)b, &prop}, p, xs + d0, ys + d0, L,
                       kBatchChunk, resident, sdata, N, tbase, nullptr, nullptr, ts);
    } else {
      trace_group<PPT>(PriorDraw{p, seed, (uint32_t)b}, p, xs + d0, ys + d0, L, kBatchChunk,
                       resident, sdata, N, tbase, nullptr, nullptr, ts);
    }
    // each warp leaves its per-degree partials of this tile in the tile's slot
    // and raises the instance's running maxima; no block-level merge per tile
    {
      const int64_t slot0 = ((int64_t)first[b] + items[it].tile) * kWarpParts + warp * kMaxDegrees;
      __syncwarp();
      if (lane < kMaxDegrees * 4) {
        const float4* src = reinterpret_cast<const float4*>(&ts.wrun[warp * kMaxDegrees]);
        reinterpret_cast<float4*>(parts + slot0)[lane] = src[lane];
      }
      if (lane < kMaxDegrees) {
        const float m = ts.wrun[warp * kMaxDegrees + lane].m;
        if (m > -INFINITY) atomicMax(inst_max + (int64_t)b * kMaxDegrees + lane, float_key(m));
      }
      __syncwarp();
      if (lane < kMaxDegrees) deg_empty(ts.wrun[warp * kMaxDegrees + lane]);
      if (tid < kMaxDegrees) ts.ext_max[tid] = -INFINITY;
    }
    if (tid == 0 && ts.nan) record_status(&hdr->status, PPL_ENAN);
    // the last item of the instance merges the instance's partials; the
    // barrier and thread 0's fence order every warp's partial writes before
    // the count (fences are cumulative)
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      last_sh = atomicSub(&count[b], 1) == 1;
    }
    __syncthreads();
    if (last_sh) {
      __threadfence();
      const int64_t i0 = first[b];
      const int64_t ni = (N + (int64_t)kTpb * PPT - 1) / ((int64_t)kTpb * PPT);
      const int64_t np = ni * (kTpb / 32);  // (tile, warp) partials per degree
      if (warp < kMaxDegrees) {
        DegPartial a;
        DegSums ds;
        merge_degree(parts + i0 * (kTpb / 32) * kMaxDegrees, (int)np, warp, lane, a, ds);
        if (lane == 0) {
          fin[warp] = a;
          fS[warp] = ds.S;
          fS2[warp] = ds.S2;
        }
      }
      __syncthreads();
      if (warp == 0)
        write_summary_warp(fin, fS, fS2, p.n_deg, p.min_deg, N,
                           lane == 0 ? ld_volatile_i32(&hdr->status) : 0, out + b);
      __syncthreads();
    }
  }
}

template <int PPT, bool LEARNED>
static cudaError_t launch_batched_t(const PolyParams& p, const float* x, const float* y,
                                    const int64_t* data_off, const int64_t* part_off,
                                    int32_t n_inst, int64_t n_items, int blocks_per_sm,
                                    uint64_t seed, const float* proposal, char* ws,
                                    ppl_is_result* out, cudaStream_t s) {
  const BatchLayout l = batch_layout(n_items, n_inst);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + l.header);
  cudaError_t e = cudaMemsetAsync(ws + l.header, 0, 512, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(ws + l.count, ws + l.count_tmpl, (size_t)n_inst * sizeof(int32_t),
                      cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(ws + l.inst_max, 0, (size_t)n_inst * kMaxDegrees * sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  const size_t smem = trace_smem_bytes<PPT>() + kBatchChunk * sizeof(float2);
  int unused = 0;
  e = device_once((const void*)batched_kernel<PPT, LEARNED>, &unused, [smem](int*) {
    return cudaFuncSetAttribute(batched_kernel<PPT, LEARNED>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel<PPT, LEARNED>, kTpb,
                                                    smem);
  if (e != cudaSuccess) return e;
  const int bps = std::max(1, std::min(blocks_per_sm, std::max(1, per_sm)));
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(n_items, (int64_t)num_sms() * bps));
  batched_kernel<PPT, LEARNED><<<(unsigned)grid, kTpb, smem, s>>>(
      p, x, y, data_off, part_off, reinterpret_cast<const BatchItem*>(ws + l.items), n_items,
      reinterpret_cast<const int32_t*>(ws + l.first), reinterpret_cast<int32_t*>(ws + l.count),
      seed, proposal, reinterpret_cast<unsigned*>(ws + l.inst_max), hdr,
      reinterpret_cast<DegPartial*>(ws + l.parts), out);
  return cudaGetLastError();
}

cudaError_t launch_batched(const PolyParams& p, const float* x, const float* y,
                           const int64_t* data_off, const int64_t* part_off, int32_t n_inst,
                           int64_t n_items, int ppt, int blocks_per_sm, uint64_t seed,
                           const float* proposal, char* ws, ppl_is_result* out, cudaStream_t s) {
#define PPL_BATCHED_CASE(P)                                                                   \
  case P:                                                                                     \
    return proposal ? launch_batched_t<P, true>(p, x, y, data_off, part_off, n_inst, n_items, \
                                                blocks_per_sm, seed, proposal, ws, out, s)    \
                    : launch_batched_t<P, false>(p, x, y, data_off, part_off, n_inst,         \
                                                 n_items, blocks_per_sm, seed, nullptr, ws,   \
                                                 out, s);
  switch (ppt) {
    PPL_BATCHED_CASE(1)
    PPL_BATCHED_CASE(2)
    PPL_BATCHED_CASE(4)
    PPL_BATCHED_CASE(8)
    default: return cudaErrorInvalidValue;
  }
#undef PPL_BATCHED_CASE
}

// Host plan.  Items are issued in rounds: round r holds tile r of every
// instance with more than r tiles, heaviest (longest data) first.  An
// instance's first tile thus finishes early and its maxima let the later
// tiles skip negligible traces; within a round the heaviest-first order keeps
// the blocks finishing together.  first[b] is instance b's base among the
// per-tile partial slots (contiguous per instance); count[b] its tile count.
static int64_t build_plan(const int64_t* data_off, const int64_t* part_off, int32_t n_inst,
                          int ppt, std::vector<BatchItem>* items, std::vector<int32_t>* first,
                          std::vector<int32_t>* count, int64_t* max_len, double* work) {
  const int64_t tile = (int64_t)kTpb * ppt;
  std::vector<int32_t> order(n_inst);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return (data_off[a + 1] - data_off[a]) > (data_off[b + 1] - data_off[b]);
  });
  items->clear();
  first->assign(n_inst, 0);
  count->assign(n_inst, 0);
  *max_len = 0;
  *work = 0.0;
  int64_t slots = 0, max_tiles = 0;
  for (int32_t b = 0; b < n_inst; ++b) {
    const int64_t L = data_off[b + 1] - data_off[b];
    const int64_t N = part_off[b + 1] - part_off[b];
    const int64_t tiles = (N + tile - 1) / tile;
    (*first)[b] = (int32_t)slots;
    (*count)[b] = (int32_t)tiles;
    slots += tiles;
    max_tiles = std::max(max_tiles, tiles);
    *max_len = std::max(*max_len, L);
    *work += (double)N * (double)L;
  }
  for (int64_t r = 0; r < max_tiles; ++r)
    for (int32_t b : order)
      if (r < (*count)[b]) items->push_back(BatchItem{b, (int32_t)r});
  return (int64_t)items->size();
}

static bool valid_offsets(const int64_t* data_off, const int64_t* part_off, int32_t n_inst) {
  if (!data_off || !part_off || n_inst < 1) return false;
  if (data_off[0] != 0 || part_off[0] != 0) return false;
  for (int32_t b = 0; b < n_inst; ++b) {
    const int64_t L = data_off[b + 1] - data_off[b], N = part_off[b + 1] - part_off[b];
    if (L < 0 || N < 1 || N > 0x7fffffffll) return false;
  }
  return true;
}

}  // namespace ppl

using namespace ppl;

namespace {

ppl_status poly_params_b(const ppl_model* m, PolyParams* p) {
  if (!m || m->id != PPL_MODEL_POLY) return PPL_EINVAL;
  const int n_deg = m->max_deg - m->min_deg + 1;
  if (m->min_deg < 0 || n_deg < 1 || n_deg > kMaxDegrees || m->coef_offset < 0 ||
      m->max_deg + m->coef_offset > kMaxCoef || !(m->obs_sigma > 0.0f))
    return PPL_EINVAL;
  p->min_deg = m->min_deg;
  p->n_deg = n_deg;
  p->coef_offset = m->coef_offset;
  p->prior_sigma = m->prior_sigma;
  p->neg_half_inv_var = (float)(-1.0 / (2.0 * (double)m->obs_sigma * (double)m->obs_sigma));
  return PPL_OK;
}

bool valid_ppt(int ppt) { return ppt == 1 || ppt == 2 || ppt == 4 || ppt == 8; }

}  // namespace

extern "C" {

size_t ppl_batched_workspace_size(const int64_t* data_off_host, const int64_t* part_off_host,
                                  int32_t n_inst, int32_t ppt) {
  if (!valid_offsets(data_off_host, part_off_host, n_inst) || !valid_ppt(ppt)) return 0;
  std::vector<BatchItem> items;
  std::vector<int32_t> first, count;
  int64_t max_len;
  double work;
  const int64_t n_items =
      build_plan(data_off_host, part_off_host, n_inst, ppt, &items, &first, &count, &max_len,
                 &work);
  // the largest plan of any candidate configuration (ppt = 1 has the most items)
  std::vector<BatchItem> i1;
  const int64_t n1 = build_plan(data_off_host, part_off_host, n_inst, 1, &i1, &first, &count,
                                &max_len, &work);
  return batch_layout(std::max(n_items, n1), n_inst).total;
}

ppl_status ppl_batched_prepare(const ppl_model* model, const int64_t* data_off_host,
                               const int64_t* part_off_host, int32_t n_inst, int32_t ppt,
                               int32_t blocks_per_sm, ppl_batch_plan* plan, void* ws,
                               size_t ws_bytes, ppl_stream stream) {
  PolyParams p;
  if (poly_params_b(model, &p) != PPL_OK) return PPL_EINVAL;
  if (!plan || !ws || !valid_ppt(ppt) || blocks_per_sm < 1 || blocks_per_sm > 32)
    return PPL_EINVAL;
  if (!valid_offsets(data_off_host, part_off_host, n_inst)) return PPL_EINVAL;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return PPL_EINVAL;
  std::vector<BatchItem> items;
  std::vector<int32_t> first, count;
  int64_t max_len;
  double work;
  const int64_t n_items =
      build_plan(data_off_host, part_off_host, n_inst, ppt, &items, &first, &count, &max_len,
                 &work);
  const BatchLayout l = batch_layout(n_items, n_inst);
  if (ws_bytes < l.total) return PPL_EINVAL;
  char* base = static_cast<char*>(ws);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(base + l.items, items.data(), items.size() * sizeof(BatchItem),
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(base + l.first, first.data(), first.size() * sizeof(int32_t),
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(base + l.count_tmpl, count.data(), count.size() * sizeof(int32_t),
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return PPL_ECUDA;
  plan->ppt = ppt;
  plan->blocks_per_sm = blocks_per_sm;
  plan->n_inst = n_inst;
  plan->n_items = n_items;
  plan->max_len = max_len;
  plan->total_particles = part_off_host[n_inst];
  plan->work = work;
  return PPL_OK;
}

ppl_status ppl_infer_is_batched(const ppl_model* model, const float* x, const float* y,
                                const int64_t* data_off, const int64_t* part_off,
                                int32_t n_inst, uint64_t seed, const ppl_batch_plan* plan,
                                ppl_is_result* out_dev, void* ws, size_t ws_bytes,
                                ppl_stream stream) {
  PolyParams p;
  if (poly_params_b(model, &p) != PPL_OK) return PPL_EINVAL;
  if (!plan || !x || !y || !data_off || !part_off || !out_dev || !ws) return PPL_EINVAL;
  if (plan->n_inst != n_inst || !valid_ppt(plan->ppt)) return PPL_EINVAL;
  if (ws_bytes < batch_layout(plan->n_items, n_inst).total) return PPL_EINVAL;
  const cudaError_t e =
      launch_batched(p, x, y, data_off, part_off, n_inst, plan->n_items, plan->ppt,
                     plan->blocks_per_sm, seed, nullptr, static_cast<char*>(ws), out_dev,
                     (cudaStream_t)stream);
  return e == cudaSuccess ? PPL_OK : PPL_ECUDA;
}

ppl_status ppl_infer_is_learned(const ppl_model* model, const float* x, const float* y,
                                const int64_t* data_off, const int64_t* part_off,
                                int32_t n_inst, uint64_t seed, const ppl_batch_plan* plan,
                                const float* proposal, ppl_is_result* out_dev, void* ws,
                                size_t ws_bytes, ppl_stream stream) {
  PolyParams p;
  if (poly_params_b(model, &p) != PPL_OK || !(model->prior_sigma > 0.0f)) return PPL_EINVAL;
  int slots = 0;
  for (int k = 0; k < p.n_deg; ++k) slots += p.min_deg + k + p.coef_offset;
  if (slots > kMaxSlots) return PPL_EINVAL;
  if (!plan || !x || !y || !data_off || !part_off || !out_dev || !ws || !proposal)
    return PPL_EINVAL;
  if (plan->n_inst != n_inst || !valid_ppt(plan->ppt)) return PPL_EINVAL;
  if (ws_bytes < batch_layout(plan->n_items, n_inst).total) return PPL_EINVAL;
  const cudaError_t e =
      launch_batched(p, x, y, data_off, part_off, n_inst, plan->n_items, plan->ppt,
                     plan->blocks_per_sm, seed, proposal, static_cast<char*>(ws), out_dev,
                     (cudaStream_t)stream);
  return e == cudaSuccess ? PPL_OK : PPL_ECUDA;
}

ppl_status ppl_batched_status(const void* ws, ppl_stream stream) {
  return ppl_workspace_status(ws, stream);
}

// Autotuner: times every (ppt, blocks_per_sm) candidate on the caller's data
// (two warm-up launches, then the median of three), keeps the fastest, and
// records it in `cache_path` (a one-line JSON object keyed by the batch's
// shape).  A cached entry with the same key is reused without timing.
ppl_status ppl_batched_autotune(const ppl_model* model, const float* x, const float* y,
                                const int64_t* data_off_dev, const int64_t* part_off_dev,
                                const int64_t* data_off_host, const int64_t* part_off_host,
                                int32_t n_inst, uint64_t seed, ppl_is_result* out_dev, void* ws,
                                size_t ws_bytes, const char* cache_path, ppl_batch_plan* best,
                                ppl_stream stream) {
  if (!best || !valid_offsets(data_off_host, part_off_host, n_inst)) return PPL_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  double work = 0.0;
  int64_t max_len = 0;
  for (int32_t b = 0; b < n_inst; ++b) {
    const int64_t L = data_off_host[b + 1] - data_off_host[b];
    work += (double)(part_off_host[b + 1] - part_off_host[b]) * (double)L;
    max_len = std::max(max_len, L);
  }
  char key[160];
  snprintf(key, sizeof key, "n%d_p%lld_w%.6e_L%lld_sm%d", n_inst,
           (long long)part_off_host[n_inst], work, (long long)max_len, num_sms());
  if (cache_path) {
    FILE* f = fopen(cache_path, "r");
    if (f) {
      char line[512] = {0};
      const size_t got = fread(line, 1, sizeof line - 1, f);
      fclose(f);
      line[got] = 0;
      char k[160] = {0};
      int ppt = 0, bps = 0;
      const char* kp = strstr(line, "\"key\": \"");
      const char* pp = strstr(line, "\"ppt\": ");
      const char* bp = strstr(line, "\"blocks_per_sm\": ");
      if (kp && pp && bp && sscanf(kp + 8, "%159[^\"]", k) == 1 && sscanf(pp + 7, "%d", &ppt) == 1 &&
          sscanf(bp + 17, "%d", &bps) == 1 && strcmp(k, key) == 0 && valid_ppt(ppt)) {
        return ppl_batched_prepare(model, data_off_host, part_off_host, n_inst, ppt, bps, best,
                                   ws, ws_bytes, stream);
      }
    }
  }
  const int ppts[] = {1, 2, 4, 8};
  const int bpss[] = {1, 2, 3, 4};
  float best_ms = 1e30f;
  int best_ppt = 4, best_bps = 2;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return PPL_ECUDA;
  for (int ppt : ppts) {
    for (int bps : bpss) {
      ppl_batch_plan plan;
      ppl_status st = ppl_batched_prepare(model, data_off_host, part_off_host, n_inst, ppt, bps,
                                          &plan, ws, ws_bytes, stream);
      if (st != PPL_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
      }
      float t[3];
      for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0, s);
        st = ppl_infer_is_batched(model, x, y, data_off_dev, part_off_dev, n_inst, seed, &plan,
                                  out_dev, ws, ws_bytes, stream);
        cudaEventRecord(e1, s);
        if (st != PPL_OK || cudaEventSynchronize(e1) != cudaSuccess) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return st != PPL_OK ? st : PPL_ECUDA;
        }
        if (r >= 2) cudaEventElapsedTime(&t[r - 2], e0, e1);
      }
      std::sort(t, t + 3);
      if (t[1] < best_ms) {
        best_ms = t[1];
        best_ppt = ppt;
        best_bps = bps;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cache_path) {
    FILE* f = fopen(cache_path, "w");
    if (f) {
      fprintf(f, "{\"key\": \"%s\", \"ppt\": %d, \"blocks_per_sm\": %d, \"ms\": %.4f}\n", key,
              best_ppt, best_bps, best_ms);
      fclose(f);
    }
  }
  return ppl_batched_prepare(model, data_off_host, part_off_host, n_inst, best_ppt, best_bps,
                             best, ws, ws_bytes, stream);
}

}  // extern "C"
