// persistent.cu -- CGLS for many uneven requests in one persistent launch.
//
// Slices are independent (Sec. 3.1) and the paper splits uneven slice counts
// into chunks (Sec. 3.1, last chunk smaller).  Here requests that share a
// geometry are packed, B slices at a time, into batches; every batch runs the
// textbook CGLS of Sec. 2.1 with per-slice FP64 scalars.  One cooperative
// kernel runs every phase of every batch: layout in, initialisation, `iters`
// iterations, layout out.  Inside a phase the work is a flat list of
// (batch, block of row groups) items spread over all resident blocks, so
// large and small requests load-balance together (the SpMM phases hand them
// out in list order from a counter); phases are separated by a grid barrier.
//
// The barrier is the library's own: it spins on a generation counter with a
// time limit read from %globaltimer.  When the limit passes (or another block
// already gave up) a block records TOMO_ERR_TIMEOUT in a status word and
// returns; every other block returns at its next barrier, so the launch
// always ends.  Vectors written inside the launch are read with coherent
// loads (the matrices, never written, keep the read-only path).
#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "spmm.cuh"

namespace tomo {

namespace {

constexpr int kItemRowGroups = 8;  // row groups per work item: one per warp (finer items balance better)

struct PSlot {        // one lane of a batch
  const float *sino;  // start of the slice's sinogram (nullptr: padding)
  float *x;           // start of the slice's tomogram
  double *hist;       // &hist[z] of the request (nullable), stride hist_ld
  int32_t hist_ld, resume;
  // optional CGLS state in / out of this slice (resume != 0: read *_in)
  const float *r_in, *p_in;
  const double *g_in;
  const int32_t *f_in;
  float *r_out, *p_out;
  double *g_out;
  int32_t *f_out;
};

struct PBatch {
  const int64_t *cpA, *cpT;
  const int32_t *rlA, *rlT;
  const int2 *entA, *entT;
  Sell16View lA, lT;
  int64_t rows, cols;
  float *x, *r, *q, *p, *s;
  float *rs;                         // 16-bit values: r times 1/a(theta) of its row (the A^T operand)
  const float *scale;                // per angle 1/a(theta) (16-bit values)
  int32_t np;
  int32_t nbands;                    // 16-bit A stored as column bands: their number, else 0
  const Sell16View *bandv;           // [nbands] the bands' views
  float *partial;                    // (rows, B) sums of the bands before the last
  double *scal;                      // B x 8
  double *part_q, *part_r, *part_s;  // items x B
  int32_t itemA0, nitemA, itemT0, nitemT;
};

struct PItem {
  int32_t batch;
  int32_t pad;
  int64_t rg0, rg1;  // row groups [rg0, rg1)
};

struct GridBar {
  unsigned int count, gen;
  int status;
  int pad;
  unsigned int work[2];  // item counters of the SpMM phases (alternating; see ph_spmm)
};

struct PPlan {
  const PBatch *batches;
  const PSlot *slots;
  const PItem *itemsA, *itemsT;
  int32_t nbatch, nitemA, nitemT, iters;
  int32_t maxbands;  // A-phase steps: the most column bands of any batch (1 when none is banded)
  GridBar *bar;
  unsigned long long timeout_ns;
  int32_t skip_block;  // test hook: this block never arrives at a barrier (-1: none)
};

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier with a time limit.  Returns false when the launch must stop.
// The last block to arrive resets item counter `reset` (>= 0) before it
// releases the others.
__device__ bool grid_barrier(const PPlan &P, int reset = -1) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    GridBar *bar = P.bar;
    volatile int *status = &bar->status;
    int ok = *status == 0;
    if (ok) {
      const unsigned int g = atomicAdd(&bar->gen, 0u);
      __threadfence();
      const unsigned int arrived = atomicAdd(&bar->count, 1u);
      if (arrived == gridDim.x - 1) {
        if (reset >= 0) atomicExch(&bar->work[reset], 0u);
        atomicExch(&bar->count, 0u);
        __threadfence();
        atomicAdd(&bar->gen, 1u);
      } else {
        const unsigned long long t0 = globaltimer();
        while (atomicAdd(&bar->gen, 0u) == g) {
          if (*status != 0) {
            ok = 0;
            break;
          }
          if (globaltimer() - t0 > P.timeout_ns) {
            atomicCAS(&bar->status, 0, (int)TOMO_ERR_TIMEOUT);
            ok = 0;
            break;
          }
          __nanosleep(100);
        }
      }
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The SpMM gathers use coherent loads (kNC = false); the epilogues of this
// kernel read nothing but their own output row.
template <int B, int kFmt, bool kTrans, class Epi>
__device__ void spmm_item(const PBatch &bt, const PItem &it, const float *X, const Epi &epi, double *ss) {
  const int64_t w = threadIdx.x >> 5;
  if constexpr (kFmt == 0) {
    if (kTrans)
      sell_rowgroups<B, Epi, false>(bt.cpT, bt.rlT, bt.entT, bt.cols, X, epi, it.rg0 + w, kWarps, it.rg1, ss);
    else
      sell_rowgroups<B, Epi, false>(bt.cpA, bt.rlA, bt.entA, bt.rows, X, epi, it.rg0 + w, kWarps, it.rg1, ss);
  } else {
    constexpr bool kBf16 = kFmt == 1;
    if (kTrans)  // X is the pre-scaled operand rs: no per-entry scale
      sell16_rowgroups<B, kBf16, true, Epi, false, true>(bt.lT, bt.cols, X, epi, it.rg0 + w, kWarps, it.rg1, ss);
    else
      sell16_rowgroups<B, kBf16, false, Epi, false>(bt.lA, bt.rows, X, epi, it.rg0 + w, kWarps, it.rg1, ss);
  }
}

// sum of one slice's partials over a batch's items, in item order (block-wide)
__device__ double batch_sum(const double *part, int nitem, int B, int s) {
  __shared__ double red[kThreads];
  double a = 0.0;
  for (int i = threadIdx.x; i < nitem; i += blockDim.x) a += part[(int64_t)i * B + s];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int o = kThreads / 2; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// Each phase is its own non-inlined function: the kernel's register budget is
// then set by the busiest phase (an SpMM) rather than by everything the
// phases would keep live across each other if inlined into one body.

// layout in: fresh slices r = b (the sinogram), x = 0; resumed slices x, r, p
// from the caller
template <int B>
__device__ __noinline__ void ph_layout_in(const PPlan &P) {
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  for (int bi = 0; bi < P.nbatch; ++bi) {
    const PBatch &bt = P.batches[bi];
    const PSlot *sl = P.slots + (int64_t)bi * B;
    for (int64_t e = gtid; e < bt.rows * B; e += gthreads) {
      const int64_t i = e / B;
      const int s = (int)(e % B);
      const float v = sl[s].resume ? sl[s].r_in[i] : (sl[s].sino ? sl[s].sino[i] : 0.f);
      bt.r[e] = v;
      if (bt.rs) bt.rs[e] = v * bt.scale[i / bt.np];
    }
    for (int64_t e = gtid; e < bt.cols * B; e += gthreads) {
      const int64_t j = e / B;
      const int s = (int)(e % B);
      bt.x[e] = sl[s].resume ? sl[s].x[j] : 0.f;
      if (sl[s].resume) bt.p[e] = sl[s].p_in[j];
    }
  }
}

// Next item of an SpMM phase, taken in order from counter `slot`: the blocks
// then stay together in the item list, so the images that the items in flight
// gather belong to one or two batches and stay in L2 (with a fixed stride, a
// block slowed by longer items falls behind and the items in flight spread
// over many batches).
__device__ __forceinline__ int next_item(const PPlan &P, int slot) {
  __shared__ int s_it;
  __syncthreads();  // every thread has read the previous item's index
  if (threadIdx.x == 0) s_it = (int)atomicAdd(&P.bar->work[slot], 1u);
  __syncthreads();
  return s_it;
}

// SpMM over every batch's items: out = M X with per-item norm partials;
// kTrans: A^T (T items, X = r, out = s) else A (A items, X = p, out = q)
template <int B, int kFmt, bool kTrans>
__device__ __noinline__ void ph_spmm(const PPlan &P, int slot) {
  constexpr int V = Lanes<B>::V, L = Lanes<B>::L;
  const int lane_s0 = ((threadIdx.x & 31) % L) * V;
  const int nitem = kTrans ? P.nitemT : P.nitemA;
  for (int it = next_item(P, slot); it < nitem; it = next_item(P, slot)) {
    const PItem &item = kTrans ? P.itemsT[it] : P.itemsA[it];
    const PBatch &bt = P.batches[item.batch];
    double ss[V];
#pragma unroll
    for (int t = 0; t < V; ++t) ss[t] = 0.0;
    if constexpr (kTrans) {
      spmm_item<B, kFmt, true>(bt, item, kFmt == 0 ? bt.r : bt.rs, EpiStoreNorm{bt.s, B}, ss);
      block_norms_to<V>(ss, lane_s0, B, bt.part_s + (int64_t)(it - bt.itemT0) * B);
    } else {
      spmm_item<B, kFmt, false>(bt, item, bt.p, EpiStoreNorm{bt.q, B}, ss);
      block_norms_to<V>(ss, lane_s0, B, bt.part_q + (int64_t)(it - bt.itemA0) * B);
    }
  }
}

// q = A p with ||q||^2, step `band` of the A phase.  A batch whose 16-bit A is
// stored as column bands runs band `band` (each step is separated by a grid
// barrier, so that every block works on the same band of the images, which
// can stay in L2): the bands before the last add their sums into the batch's
// partial buffer, the last adds it and stores q with the norm partials.  Other
// batches run whole at step 0.
template <int B, int kFmt>
__device__ __noinline__ void ph_spmm_a(const PPlan &P, int band, int slot) {
  constexpr int V = Lanes<B>::V, L = Lanes<B>::L;
  const int lane_s0 = ((threadIdx.x & 31) % L) * V;
  for (int it = next_item(P, slot); it < P.nitemA; it = next_item(P, slot)) {
    const PItem &item = P.itemsA[it];
    const PBatch &bt = P.batches[item.batch];
    const int nb = bt.nbands;
    if (nb == 0 ? band != 0 : band >= nb) continue;  // uniform over the block (one item per block)
    double ss[V];
#pragma unroll
    for (int t = 0; t < V; ++t) ss[t] = 0.0;
    if constexpr (kFmt != 0) {
      if (nb > 0) {
        constexpr bool kBf16 = kFmt == 1;
        const Sell16View v = bt.bandv[band];
        const int64_t w = threadIdx.x >> 5;
        if (band < nb - 1) {
          sell16_rowgroups<B, kBf16, false, EpiBandPartial, false>(v, bt.rows, bt.p,
                                                                   EpiBandPartial{bt.partial, B, band == 0},
                                                                   item.rg0 + w, kWarps, item.rg1, ss);
          continue;
        }
        sell16_rowgroups<B, kBf16, false, EpiBandLast<EpiStoreNorm>, false>(
            v, bt.rows, bt.p, EpiBandLast<EpiStoreNorm>{bt.partial, B, EpiStoreNorm{bt.q, B}}, item.rg0 + w, kWarps,
            item.rg1, ss);
        block_norms_to<V>(ss, lane_s0, B, bt.part_q + (int64_t)(it - bt.itemA0) * B);
        continue;
      }
    }
    spmm_item<B, kFmt, false>(bt, item, bt.p, EpiStoreNorm{bt.q, B}, ss);
    block_norms_to<V>(ss, lane_s0, B, bt.part_q + (int64_t)(it - bt.itemA0) * B);
  }
}

// gamma = ||s||^2 (resumed slices: gamma, frozen from the state), p = s
template <int B>
__device__ __noinline__ void ph_init_scalars(const PPlan &P) {
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  for (int pr = blockIdx.x; pr < P.nbatch * B; pr += gridDim.x) {
    const PBatch &bt = P.batches[pr / B];
    const int s = pr % B;
    const PSlot &sl = P.slots[pr];
    const double g = batch_sum(bt.part_s, bt.nitemT, B, s);
    if (threadIdx.x == 0) {
      bt.scal[s * 8 + 0] = sl.resume ? *sl.g_in : g;
      bt.scal[s * 8 + 1] = 0.0;
      bt.scal[s * 8 + 2] = 0.0;
      bt.scal[s * 8 + 3] = sl.resume ? (*sl.f_in != 0 ? 1.0 : 0.0) : (g == 0.0 ? 1.0 : 0.0);
    }
  }
  for (int bi = 0; bi < P.nbatch; ++bi) {
    const PBatch &bt = P.batches[bi];
    const PSlot *sl = P.slots + (int64_t)bi * B;
    for (int64_t e = gtid; e < bt.cols * B; e += gthreads)
      if (!sl[e % B].resume) bt.p[e] = bt.s[e];
  }
}

// alpha = gamma / ||q||^2
template <int B>
__device__ __noinline__ void ph_alpha(const PPlan &P) {
  for (int pr = blockIdx.x; pr < P.nbatch * B; pr += gridDim.x) {
    const PBatch &bt = P.batches[pr / B];
    const int s = pr % B;
    const double qq = batch_sum(bt.part_q, bt.nitemA, B, s);
    if (threadIdx.x == 0) {
      const double gam = bt.scal[s * 8 + 0];
      const bool frozen = bt.scal[s * 8 + 3] != 0.0 || gam == 0.0 || qq == 0.0;
      bt.scal[s * 8 + 3] = frozen ? 1.0 : 0.0;
      bt.scal[s * 8 + 1] = frozen ? 0.0 : gam / qq;
    }
  }
}

// r -= alpha q (A items, ||r||^2 partials); x += alpha p (T items)
template <int B>
__device__ __noinline__ void ph_step(const PPlan &P) {
  constexpr int V = Lanes<B>::V, G = Lanes<B>::G, PER = B / V;
  for (int it = blockIdx.x; it < P.nitemA + P.nitemT; it += gridDim.x) {
    const bool onA = it < P.nitemA;
    const PItem &item = onA ? P.itemsA[it] : P.itemsT[it - P.nitemA];
    const PBatch &bt = P.batches[item.batch];
    const int64_t n = onA ? bt.rows : bt.cols;
    const int64_t e0 = item.rg0 * G * PER, e1 = std::min<int64_t>(item.rg1 * G, n) * PER;  // vector indices
    // this thread's slice offset is fixed: kThreads is a multiple of PER
    const int s0 = (int)((threadIdx.x % PER) * V);
    float al[V];
#pragma unroll
    for (int t = 0; t < V; ++t) al[t] = (float)bt.scal[(s0 + t) * 8 + 1];
    double ss[V];
#pragma unroll
    for (int t = 0; t < V; ++t) ss[t] = 0.0;
    for (int64_t i = e0 + threadIdx.x; i < e1; i += blockDim.x) {
      if (onA) {
        Vec<V> rv = ld_vec<V>(bt.r + i * V), qv = ld_vec<V>(bt.q + i * V);
#pragma unroll
        for (int t = 0; t < V; ++t) {
          rv.v[t] = fmaf(-al[t], qv.v[t], rv.v[t]);
          ss[t] += (double)rv.v[t] * (double)rv.v[t];
        }
        st_vec<V>(bt.r + i * V, rv);
        if (bt.rs) {  // the A^T operand: row i / PER, angle (i / PER) / np
          const float sc = bt.scale[(i / PER) / bt.np];
#pragma unroll
          for (int t = 0; t < V; ++t) rv.v[t] *= sc;
          st_vec<V>(bt.rs + i * V, rv);
        }
      } else {
        Vec<V> xv = ld_vec<V>(bt.x + i * V), pv = ld_vec<V>(bt.p + i * V);
#pragma unroll
        for (int t = 0; t < V; ++t) xv.v[t] = fmaf(al[t], pv.v[t], xv.v[t]);
        st_vec<V>(bt.x + i * V, xv);
      }
    }
    if (onA) block_norms_to<V>(ss, s0, B, bt.part_r + (int64_t)(it - bt.itemA0) * B);
  }
}

// beta = gamma'/gamma, residual history
template <int B>
__device__ __noinline__ void ph_beta(const PPlan &P, int iter) {
  for (int pr = blockIdx.x; pr < P.nbatch * B; pr += gridDim.x) {
    const PBatch &bt = P.batches[pr / B];
    const int s = pr % B;
    const double gs = batch_sum(bt.part_s, bt.nitemT, B, s);
    const double rr = batch_sum(bt.part_r, bt.nitemA, B, s);
    if (threadIdx.x == 0) {
      if (bt.scal[s * 8 + 3] != 0.0) {
        bt.scal[s * 8 + 2] = 0.0;
      } else {
        bt.scal[s * 8 + 2] = gs / bt.scal[s * 8 + 0];
        bt.scal[s * 8 + 0] = gs;
      }
      const PSlot &sl = P.slots[pr];
      if (sl.sino && sl.hist) sl.hist[(int64_t)iter * sl.hist_ld] = sqrt(rr);
    }
  }
}

// p = s + beta p
template <int B>
__device__ __noinline__ void ph_direction(const PPlan &P) {
  constexpr int V = Lanes<B>::V, G = Lanes<B>::G, PER = B / V;
  for (int it = blockIdx.x; it < P.nitemT; it += gridDim.x) {
    const PItem &item = P.itemsT[it];
    const PBatch &bt = P.batches[item.batch];
    const int64_t e0 = item.rg0 * G * PER, e1 = std::min<int64_t>(item.rg1 * G, bt.cols) * PER;
    const int s0 = (int)((threadIdx.x % PER) * V);
    float be[V];
#pragma unroll
    for (int t = 0; t < V; ++t) be[t] = (float)bt.scal[(s0 + t) * 8 + 2];
    for (int64_t i = e0 + threadIdx.x; i < e1; i += blockDim.x) {
      Vec<V> pv = ld_vec<V>(bt.p + i * V), sv = ld_vec<V>(bt.s + i * V);
#pragma unroll
      for (int t = 0; t < V; ++t) pv.v[t] = fmaf(be[t], pv.v[t], sv.v[t]);
      st_vec<V>(bt.p + i * V, pv);
    }
  }
}

// layout out: x (and the state, where asked) to the requests
template <int B>
__device__ __noinline__ void ph_layout_out(const PPlan &P) {
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  for (int bi = 0; bi < P.nbatch; ++bi) {
    const PBatch &bt = P.batches[bi];
    const PSlot *sl = P.slots + (int64_t)bi * B;
    for (int64_t e = gtid; e < bt.cols * B; e += gthreads) {
      const int64_t j = e / B;
      const int s = (int)(e % B);
      if (sl[s].sino) sl[s].x[j] = bt.x[e];
      if (sl[s].p_out) sl[s].p_out[j] = bt.p[e];
    }
    for (int64_t e = gtid; e < bt.rows * B; e += gthreads) {
      const int s = (int)(e % B);
      if (sl[s].r_out) sl[s].r_out[e / B] = bt.r[e];
    }
    for (int64_t s = gtid; s < B; s += gthreads) {
      if (sl[s].g_out) *sl[s].g_out = bt.scal[s * 8 + 0];
      if (sl[s].f_out) *sl[s].f_out = bt.scal[s * 8 + 3] != 0.0 ? 1 : 0;
    }
  }
}

// Five resident blocks per SM, the occupancy of the stand-alone SELL kernels
// (48 registers; the SpMM phase spills under 100 bytes, and the launch ran
// 1.27x faster than at 64 registers and four blocks).
template <int B, int kFmt>
__global__ void __launch_bounds__(kThreads, 5) k_cgls_persistent(PPlan P) {
  if ((int)blockIdx.x == P.skip_block) return;  // test hook: a block that never arrives
  int slot = 0;  // item counter of the next SpMM phase; the barrier after it resets the other
  ph_layout_in<B>(P);
  if (!grid_barrier(P)) return;
  ph_spmm<B, kFmt, true>(P, slot);  // s = A^T r, ||s||^2
  if (!grid_barrier(P, slot ^ 1)) return;
  slot ^= 1;
  ph_init_scalars<B>(P);  // gamma, p = s
  if (!grid_barrier(P)) return;
  for (int iter = 0; iter < P.iters; ++iter) {
    for (int band = 0; band < P.maxbands; ++band) {  // q = A p, ||q||^2
      ph_spmm_a<B, kFmt>(P, band, slot);
      if (!grid_barrier(P, slot ^ 1)) return;
      slot ^= 1;
    }
    ph_alpha<B>(P);
    if (!grid_barrier(P)) return;
    ph_step<B>(P);  // r -= alpha q, x += alpha p
    if (!grid_barrier(P)) return;
    ph_spmm<B, kFmt, true>(P, slot);  // s = A^T r, ||s||^2
    if (!grid_barrier(P, slot ^ 1)) return;
    slot ^= 1;
    ph_beta<B>(P, iter);
    if (!grid_barrier(P)) return;
    ph_direction<B>(P);  // p = s + beta p
    if (!grid_barrier(P)) return;
  }
  ph_layout_out<B>(P);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Layout {
  struct Batch {
    const tomo_matrix *h;
    int cnt;
    std::vector<PSlot> slots;
  };
  std::vector<Batch> batches;
  std::vector<PItem> itemsA, itemsT;
  std::vector<int32_t> itemA0, itemT0;
  size_t bytes = 0;
};

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

tomo_status plan_layout(const tomo_request *reqs, int32_t n, int B, bool pre, Layout *L) {
  // group requests by geometry handle, in order of first appearance
  std::vector<const tomo_matrix *> order;
  std::map<const tomo_matrix *, std::vector<int>> groups;
  for (int i = 0; i < n; ++i) {
    if (!groups.count(reqs[i].A)) order.push_back(reqs[i].A);
    groups[reqs[i].A].push_back(i);
  }
  for (const tomo_matrix *h : order) {
    Layout::Batch cur{h, 0, {}};
    for (int ri : groups[h]) {
      const tomo_request &q = reqs[ri];
      for (int z = 0; z < q.n_z; ++z) {
        PSlot sl;
        std::memset(&sl, 0, sizeof(sl));
        sl.sino = q.sino + (int64_t)z * h->A.rows;
        sl.x = q.x + (int64_t)z * h->A.cols;
        sl.hist = q.resnorm_hist ? q.resnorm_hist + z : nullptr;
        sl.hist_ld = q.n_z;
        if (q.state_in) {
          sl.resume = 1;
          sl.r_in = q.state_in->r + (int64_t)z * h->A.rows;
          sl.p_in = q.state_in->p + (int64_t)z * h->A.cols;
          sl.g_in = q.state_in->gamma + z;
          sl.f_in = q.state_in->frozen + z;
        }
        if (q.state_out) {
          sl.r_out = q.state_out->r + (int64_t)z * h->A.rows;
          sl.p_out = q.state_out->p + (int64_t)z * h->A.cols;
          sl.g_out = q.state_out->gamma + z;
          sl.f_out = q.state_out->frozen + z;
        }
        cur.slots.push_back(sl);
        if ((int)cur.slots.size() == B) {
          cur.cnt = B;
          L->batches.push_back(cur);
          cur = Layout::Batch{h, 0, {}};
        }
      }
    }
    if (!cur.slots.empty()) {
      cur.cnt = (int)cur.slots.size();
      PSlot pad;
      std::memset(&pad, 0, sizeof(pad));
      while ((int)cur.slots.size() < B) cur.slots.push_back(pad);
      L->batches.push_back(cur);
    }
  }
  const int G = 32 / (B / (B >= 4 ? 4 : B));
  size_t bytes = 0;
  for (size_t bi = 0; bi < L->batches.size(); ++bi) {
    const tomo_matrix *h = L->batches[bi].h;
    const int64_t rows = h->A.rows, cols = h->A.cols;
    const int64_t rgA = (rows + G - 1) / G, rgT = (cols + G - 1) / G;
    L->itemA0.push_back((int32_t)L->itemsA.size());
    for (int64_t rg = 0; rg < rgA; rg += kItemRowGroups)
      L->itemsA.push_back(PItem{(int32_t)bi, 0, rg, std::min<int64_t>(rg + kItemRowGroups, rgA)});
    L->itemT0.push_back((int32_t)L->itemsT.size());
    for (int64_t rg = 0; rg < rgT; rg += kItemRowGroups)
      L->itemsT.push_back(PItem{(int32_t)bi, 0, rg, std::min<int64_t>(rg + kItemRowGroups, rgT)});
    const int64_t nA = L->itemsA.size() - L->itemA0.back(), nT = L->itemsT.size() - L->itemT0.back();
    if (pre && !h->lpAb.empty())  // band views and the bands' partial sums
      bytes += align256(sizeof(Sell16View) * h->lpAb.size()) + align256(sizeof(float) * rows * B);
    bytes += (pre ? 3 : 2) * align256(sizeof(float) * rows * B) + 3 * align256(sizeof(float) * cols * B) +
             align256(sizeof(double) * B * 8) + 2 * align256(sizeof(double) * nA * B) +
             align256(sizeof(double) * nT * B);
  }
  bytes += align256(sizeof(PBatch) * L->batches.size()) + align256(sizeof(PSlot) * L->batches.size() * B) +
           align256(sizeof(PItem) * L->itemsA.size()) + align256(sizeof(PItem) * L->itemsT.size()) +
           align256(sizeof(GridBar));
  L->bytes = bytes;
  return TOMO_OK;
}

tomo_status check_requests(const tomo_request *reqs, int32_t n, int B, int fmt) {
  if (!reqs || n < 1) return fail(TOMO_ERR_INVALID_ARG, "need at least one request");
  if (B != 4 && B != 8 && B != 16 && B != 32) return fail(TOMO_ERR_UNSUPPORTED, "batched CGLS needs width 4, 8, 16 or 32");
  if (fmt != TOMO_FMT_SELL && fmt != TOMO_FMT_SELL16)
    return fail(TOMO_ERR_UNSUPPORTED, "batched CGLS streams TOMO_FMT_SELL or TOMO_FMT_SELL16");
  int dev = -1, lp = -2;
  for (int i = 0; i < n; ++i) {
    const tomo_request &q = reqs[i];
    if (!q.A || !q.sino || !q.x || q.n_z < 1) return fail(TOMO_ERR_INVALID_ARG, "request with a NULL pointer or n_z < 1");
    if (((uintptr_t)q.sino & 15u) || ((uintptr_t)q.x & 15u))
      return fail(TOMO_ERR_INVALID_ARG, "request buffers must be 16-byte aligned");
    for (const tomo_cgls_state *s : {q.state_in, (const tomo_cgls_state *)q.state_out})
      if (s && (!s->r || !s->p || !s->gamma || !s->frozen))
        return fail(TOMO_ERR_INVALID_ARG, "a request's CGLS state has a NULL buffer");
    if (dev < 0) dev = q.A->device;
    if (q.A->device != dev) return fail(TOMO_ERR_INVALID_ARG, "all requests must live on one device");
    if (fmt == TOMO_FMT_SELL && !q.A->sA.ent)
      return fail(TOMO_ERR_UNSUPPORTED, "a matrix was built without the FP32 SELL form");
    if (fmt == TOMO_FMT_SELL16) {
      if (q.A->lp_dtype == TOMO_F32) return fail(TOMO_ERR_UNSUPPORTED, "a matrix was built without 16-bit values");
      if (lp == -2) lp = q.A->lp_dtype;
      if (q.A->lp_dtype != lp) return fail(TOMO_ERR_UNSUPPORTED, "requests mix bf16 and f16 matrices");
    }
  }
  return TOMO_OK;
}

template <int B, int kFmt>
tomo_status launch_persistent(PPlan plan, cudaStream_t st) {
  static int res = 0;
  if (!res) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res, k_cgls_persistent<B, kFmt>, kThreads, 0) !=
            cudaSuccess ||
        res <= 0) {
      cudaGetLastError();
      return fail(TOMO_ERR_CUDA, "occupancy query for the persistent kernel failed");
    }
  }
  dim3 grid(num_sms() * res), block(kThreads);
  void *args[] = {&plan};
  TOMO_CUDA(cudaLaunchCooperativeKernel((void *)k_cgls_persistent<B, kFmt>, grid, block, args, 0, st));
  return TOMO_OK;
}

template <int B>
tomo_status launch_fmt(PPlan plan, int fmt, int lp_dtype, cudaStream_t st) {
  if (fmt == TOMO_FMT_SELL) return launch_persistent<B, 0>(plan, st);
  return lp_dtype == TOMO_BF16 ? launch_persistent<B, 1>(plan, st) : launch_persistent<B, 2>(plan, st);
}

}  // namespace

tomo_status batched_workspace(const tomo_request *reqs, int32_t n, const tomo_exec_opts *o, size_t *bytes) {
  const int B = o && o->batch_width ? o->batch_width : 16;
  const int fmt = o ? o->format : TOMO_FMT_SELL;
  TOMO_TRY(check_requests(reqs, n, B, fmt));
  Layout L;
  TOMO_TRY(plan_layout(reqs, n, B, fmt == TOMO_FMT_SELL16, &L));
  *bytes = L.bytes;
  return TOMO_OK;
}

tomo_status run_cgls_batched(const tomo_request *reqs, int32_t n, int32_t iters, const tomo_exec_opts *o,
                             void *ws, size_t ws_bytes, cudaStream_t st) {
  const int B = o && o->batch_width ? o->batch_width : 16;
  const int fmt = o ? o->format : TOMO_FMT_SELL;
  TOMO_TRY(check_requests(reqs, n, B, fmt));
  if (iters < 0) return fail(TOMO_ERR_INVALID_ARG, "iters must be >= 0");
  Layout L;
  TOMO_TRY(plan_layout(reqs, n, B, fmt == TOMO_FMT_SELL16, &L));
  void *own = nullptr;
  if (!ws) {
    cudaError_t e = cudaMallocAsync(&own, L.bytes, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(TOMO_ERR_OOM, "workspace allocation of " + std::to_string(L.bytes) + " bytes failed");
    }
    ws = own;
  } else if (ws_bytes < L.bytes) {
    return fail(TOMO_ERR_INVALID_ARG, "workspace too small: need " + std::to_string(L.bytes));
  }
  struct Free {
    void *p;
    cudaStream_t s;
    ~Free() {
      if (p) cudaFreeAsync(p, s);
    }
  } guard{own, st};

  char *base = (char *)ws;
  size_t off = 0;
  auto take = [&](size_t nbytes) {
    void *r = base + off;
    off += align256(nbytes);
    return r;
  };
  std::vector<PBatch> hb(L.batches.size());
  std::vector<PSlot> hs;
  int32_t maxbands = 1;
  for (size_t bi = 0; bi < L.batches.size(); ++bi) {
    const tomo_matrix *h = L.batches[bi].h;
    PBatch &b = hb[bi];
    std::memset(&b, 0, sizeof(b));
    b.cpA = h->sA.cp;
    b.rlA = h->sA.rl;
    b.entA = h->sA.ent;
    b.cpT = h->sAT.cp;
    b.rlT = h->sAT.rl;
    b.entT = h->sAT.ent;
    const float inv_np = 1.0f / (float)h->np;
    b.lA = Sell16View{h->lpA.cpw, h->lpA.cpb, h->lpA.rl, h->lpA.ow, h->lpA.base, h->ang_scale, h->np, inv_np,
                      h->lpA.nb4};
    b.lT = Sell16View{h->lpAT.cpw, h->lpAT.cpb, h->lpAT.rl, h->lpAT.ow, h->lpAT.base, h->ang_scale, h->np, inv_np};
    b.rows = h->A.rows;
    b.cols = h->A.cols;
    b.itemA0 = L.itemA0[bi];
    b.itemT0 = L.itemT0[bi];
    b.nitemA = (int32_t)((bi + 1 < L.batches.size() ? L.itemA0[bi + 1] : (int32_t)L.itemsA.size()) - b.itemA0);
    b.nitemT = (int32_t)((bi + 1 < L.batches.size() ? L.itemT0[bi + 1] : (int32_t)L.itemsT.size()) - b.itemT0);
    b.r = (float *)take(sizeof(float) * b.rows * B);
    b.q = (float *)take(sizeof(float) * b.rows * B);
    b.x = (float *)take(sizeof(float) * b.cols * B);
    b.p = (float *)take(sizeof(float) * b.cols * B);
    b.s = (float *)take(sizeof(float) * b.cols * B);
    if (fmt == TOMO_FMT_SELL16) {
      b.rs = (float *)take(sizeof(float) * b.rows * B);
      b.scale = h->ang_scale;
      if (!h->lpAb.empty()) {
        std::vector<Sell16View> views;
        for (const SellLp &Lb : h->lpAb)
          views.push_back(Sell16View{Lb.cpw, Lb.cpb, Lb.rl, Lb.ow, Lb.base, h->ang_scale, h->np, inv_np, Lb.nb4});
        Sell16View *dv = (Sell16View *)take(sizeof(Sell16View) * views.size());
        TOMO_CUDA(cudaMemcpyAsync(dv, views.data(), sizeof(Sell16View) * views.size(), cudaMemcpyHostToDevice, st));
        b.nbands = (int32_t)views.size();
        b.bandv = dv;
        b.partial = (float *)take(sizeof(float) * b.rows * B);
        maxbands = std::max(maxbands, b.nbands);
      }
    }
    b.np = h->np;
    b.scal = (double *)take(sizeof(double) * B * 8);
    b.part_q = (double *)take(sizeof(double) * b.nitemA * B);
    b.part_r = (double *)take(sizeof(double) * b.nitemA * B);
    b.part_s = (double *)take(sizeof(double) * b.nitemT * B);
    hs.insert(hs.end(), L.batches[bi].slots.begin(), L.batches[bi].slots.end());
  }
  PBatch *db = (PBatch *)take(sizeof(PBatch) * hb.size());
  PSlot *dsl = (PSlot *)take(sizeof(PSlot) * hs.size());
  PItem *dA = (PItem *)take(sizeof(PItem) * L.itemsA.size());
  PItem *dT = (PItem *)take(sizeof(PItem) * L.itemsT.size());
  GridBar *bar = (GridBar *)take(sizeof(GridBar));
  TOMO_CUDA(cudaMemcpyAsync(db, hb.data(), sizeof(PBatch) * hb.size(), cudaMemcpyHostToDevice, st));
  TOMO_CUDA(cudaMemcpyAsync(dsl, hs.data(), sizeof(PSlot) * hs.size(), cudaMemcpyHostToDevice, st));
  TOMO_CUDA(cudaMemcpyAsync(dA, L.itemsA.data(), sizeof(PItem) * L.itemsA.size(), cudaMemcpyHostToDevice, st));
  TOMO_CUDA(cudaMemcpyAsync(dT, L.itemsT.data(), sizeof(PItem) * L.itemsT.size(), cudaMemcpyHostToDevice, st));
  TOMO_CUDA(cudaMemsetAsync(bar, 0, sizeof(GridBar), st));

  PPlan plan;
  plan.batches = db;
  plan.slots = dsl;
  plan.itemsA = dA;
  plan.itemsT = dT;
  plan.nbatch = (int32_t)hb.size();
  plan.nitemA = (int32_t)L.itemsA.size();
  plan.nitemT = (int32_t)L.itemsT.size();
  plan.iters = iters;
  plan.maxbands = maxbands;
  plan.bar = bar;
  const double tsec = o && o->timeout_s > 0 ? o->timeout_s : 10.0;
  plan.timeout_ns = (unsigned long long)(tsec * 1e9);
  plan.skip_block = o && (o->test_flags & 1) ? 0 : -1;
  const int lp_dtype = reqs[0].A->lp_dtype;
  tomo_status s;
  switch (B) {
    case 4: s = launch_fmt<4>(plan, fmt, lp_dtype, st); break;
    case 8: s = launch_fmt<8>(plan, fmt, lp_dtype, st); break;
    case 16: s = launch_fmt<16>(plan, fmt, lp_dtype, st); break;
    default: s = launch_fmt<32>(plan, fmt, lp_dtype, st); break;
  }
  TOMO_TRY(s);
  if (o && o->async) return fold_status(&bar->status, st);  // read later by tomo_stream_status
  int status = 0;
  TOMO_CUDA(cudaMemcpyAsync(&status, &bar->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  TOMO_CUDA(cudaStreamSynchronize(st));
  if (status != 0)
    return fail((tomo_status)status, "a grid barrier of the persistent CGLS launch ran past its time limit");
  return TOMO_OK;
}

}  // namespace tomo
