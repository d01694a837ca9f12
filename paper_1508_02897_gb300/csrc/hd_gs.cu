// Streaming double-single Gram-Schmidt passes of the Arnoldi step (Sec. 3 outer
// solver: each step orthogonalises w = A z_j against the basis by classical
// Gram-Schmidt, h = V^H w, then w - V h).
//
// Both passes stream the basis V (float pairs, 16 bytes per complex entry) and one
// FP64 vector once per pass, with a few FP32 operations per byte: they are bound by
// HBM if enough bytes are in flight.  Register-held loads leave too few (each warp
// has its loads outstanding only between compute phases), so here a producer warp
// moves 16 KB tiles with bulk copies into a ring of shared-memory stages, completion
// tracked by mbarriers, while eight consumer warps work on the tiles already landed.
// The CTAs are persistent (two per SM) and take work items of GS_ITEM entries of one
// right-hand side round-robin; the producer runs ahead across item boundaries, so an
// item's block reduction overlaps the next item's copies.
//
// k_gs_dots:   partial[r][k][item] = sum over the item's entries of conj(V_r[k]) w_r
//              (and ||w_r||^2 as entry nk with `self`), double-single sums combined in a
//              fixed order (deterministic); k_reduce adds the items' partials.
// k_gs_update: y_r = g_r (base_r - sum_k V_r[k] coef_r[k] sc_r[k]^2) into y_r (FP64,
//              the preconditioner's input) and into basis slot nk (float pairs), with
//              optional per-item partials of ||y_r||^2.
// Every wait is bounded; a wait that gives up sets ST_TIMEOUT in the status word and
// the CTA unwinds (the other warps see the abort flag).
#include "hd_internal.cuh"
#include "hd_tc.cuh"

namespace hd {

namespace {

constexpr int GS_CONS = 256;                  // consumer threads (8 warps)
constexpr int GS_THREADS = GS_CONS + 32;      // + one producer warp
constexpr int GS_TILE = 1024;                 // entries per ring stage (16 KB)
constexpr int GS_EPT = GS_TILE / GS_CONS;     // entries per consumer thread and tile
constexpr int GS_ITEM = 4 * GS_TILE;          // entries per work item (one partial sum each)
constexpr int GS_NS = 6;                      // ring stages: 96 KB, two CTAs per SM
constexpr int GS_CTAS_PER_SM = 2;

struct GsRing {
  float4 *ring;        // [GS_NS][GS_TILE]
  uint64_t *full, *empty;
  volatile int *abort_flag;
};

__device__ __forceinline__ void gs_bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::su32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc::su32(dst)),
               "l"(src), "r"(bytes), "r"(tc::su32(bar))
               : "memory");
}
__device__ __forceinline__ void gs_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::su32(bar)) : "memory");
}
__device__ __forceinline__ void gs_consumer_sync() { asm volatile("bar.sync 1, %0;" ::"r"(GS_CONS) : "memory"); }

// Shared memory: the ring, then the barriers and the abort flag.
__device__ __forceinline__ GsRing gs_ring(unsigned char *smem) {
  GsRing g;
  g.ring = reinterpret_cast<float4 *>(smem);
  g.full = reinterpret_cast<uint64_t *>(smem + (size_t)GS_NS * GS_TILE * sizeof(float4));
  g.empty = g.full + GS_NS;
  g.abort_flag = reinterpret_cast<volatile int *>(g.empty + GS_NS);
  return g;
}
constexpr size_t gs_ring_bytes() { return (size_t)GS_NS * GS_TILE * sizeof(float4) + 2 * GS_NS * sizeof(uint64_t) + 16; }

__device__ __forceinline__ void gs_init(const GsRing &g) {
  if (threadIdx.x == 0) {
    for (int q = 0; q < GS_NS; ++q) {
      tc::bar_init(&g.full[q], 1);
      tc::bar_init(&g.empty[q], GS_CONS / 32);
    }
    *g.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

__device__ __forceinline__ bool gs_item_off(int r, const int *skip, const int *live) {
  return (skip && skip[r]) || (live && !live[r]);
}

// Producer: the tiles of every item of this CTA, in the consumers' order.  Tile t of a
// chunk comes from src(r, t) + chunk start; `per` tiles per chunk.
template <typename SrcFn>
__device__ __forceinline__ void gs_produce(const GsRing &g, int64_t n, int S, int T, int per, const int *skip,
                                           const int *live, int32_t *status, SrcFn src) {
  uint32_t it = 0, issued = 0;
  bool ok = true;
  for (int q = blockIdx.x; q < T && ok; q += gridDim.x) {
    const int r = q / S, seg = q - r * S;
    if (gs_item_off(r, skip, live)) continue;
    const int64_t e0 = (int64_t)seg * GS_ITEM, e1 = min(n, e0 + GS_ITEM);
    for (int64_t c0 = e0; c0 < e1 && ok; c0 += GS_TILE) {
      const uint32_t bytes = (uint32_t)(min((int64_t)GS_TILE, e1 - c0) * 16);
      for (int t = 0; t < per; ++t, ++it) {
        const int slot = (int)(it % GS_NS);
        const uint32_t ph = (it / GS_NS) & 1u;
        if (!tc::bar_wait(&g.empty[slot], ph ^ 1u, g.abort_flag)) { ok = false; break; }
        gs_bulk_g2s(g.ring + (size_t)slot * GS_TILE, src(r, t) + c0 * 16, bytes, &g.full[slot]);
        issued = it + 1;
      }
    }
  }
  if (!ok) {
    *g.abort_flag = 1;
    atomicOr(status, ST_TIMEOUT);
  }
  // no copy may still be landing in shared memory when the CTA exits
  for (uint32_t k = issued > (uint32_t)GS_NS ? issued - GS_NS : 0u; k < issued; ++k)
    tc::bar_wait(&g.full[k % GS_NS], (k / GS_NS) & 1u, g.abort_flag);
}

// Consumer side of one tile: wait for it (once per thread; a failed wait flags the abort).
__device__ __forceinline__ const float4 *gs_acquire(const GsRing &g, uint32_t it, bool &ok, int32_t *status) {
  const int slot = (int)(it % GS_NS);
  if (ok && !tc::bar_wait(&g.full[slot], (it / GS_NS) & 1u, g.abort_flag)) {
    ok = false;
    *g.abort_flag = 1;
    atomicOr(status, ST_TIMEOUT);
  }
  return g.ring + (size_t)slot * GS_TILE;
}
// Frees a tile's slot for the producer: every thread fences its shared-memory reads of
// the slot against the async proxy (the next bulk copy into the slot is an async-proxy
// write), then one lane per warp arrives.  Callers also release only after the values
// they loaded are used.  Without the fence, an arrive issued right after the loads
// became visible while a load was still outstanding, and the next copy overwrote data
// not yet read (seen as another vector's bytes, an FP64 tile read as float pairs, when a
// chunk had one more tile than the ring has stages).
__device__ __forceinline__ void gs_release(const GsRing &g, uint32_t it) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if ((threadIdx.x & 31) == 0) gs_arrive(&g.empty[it % GS_NS]);
}

}  // namespace

// ------------------------------------------------------------------ dots
// Tiles per chunk: w, then V_0 .. V_{nk0-1}.  Consumer thread t takes entries
// t + 256 u (u < 4) of every tile: w split into float pairs stays in registers for the
// chunk, each V_k tile adds to that vector's double-single accumulators.
template <int KM>
__global__ void __launch_bounds__(GS_THREADS, GS_CTAS_PER_SM)
k_gs_dots(const float4 *__restrict__ V, int64_t ldv, int64_t ldvr, int nk0, const double2 *__restrict__ w_all,
          int64_t ldw, int64_t n, int B, double2 *__restrict__ partial_all, int S, int64_t ldp,
          const int *__restrict__ skip, const int *__restrict__ live, int self, int32_t *status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ float4 red[GS_CONS / 32][KM + 1];
  const GsRing g = gs_ring(smem_raw);
  gs_init(g);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int T = B * S;
  if (warp == GS_CONS / 32) {
    if (lane == 0)
      gs_produce(g, n, S, T, nk0 + 1, skip, live, status, [&](int r, int t) -> const char * {
        return t == 0 ? reinterpret_cast<const char *>(w_all + (int64_t)r * ldw)
                      : reinterpret_cast<const char *>(V + (int64_t)r * ldvr + (int64_t)(t - 1) * ldv);
      });
    return;
  }
  uint32_t it = 0;
  bool ok = true;
  for (int q = blockIdx.x; q < T; q += gridDim.x) {
    const int r = q / S, seg = q - r * S;
    if (gs_item_off(r, skip, live)) continue;
    const int64_t e0 = (int64_t)seg * GS_ITEM, e1 = min(n, e0 + GS_ITEM);
    float acc[KM][4];
    float sh = 0.f, sl = 0.f;   // ||w||^2
#pragma unroll
    for (int k = 0; k < KM; ++k) acc[k][0] = acc[k][1] = acc[k][2] = acc[k][3] = 0.f;
    for (int64_t c0 = e0; c0 < e1; c0 += GS_TILE) {
      const int cnt = (int)min((int64_t)GS_TILE, e1 - c0);
      float4 wv[GS_EPT];
      {
        const double2 *tw = reinterpret_cast<const double2 *>(gs_acquire(g, it, ok, status));
#pragma unroll
        for (int u = 0; u < GS_EPT; ++u) {
          const int e = u * GS_CONS + tid;
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (e < cnt) {
            const double2 x = tw[e];
            const float2 a = ds_split(x.x), b = ds_split(x.y);
            v = make_float4(a.x, a.y, b.x, b.y);
          }
          wv[u] = v;
        }
        gs_release(g, it);   // after the split, which uses the loaded values
        ++it;
      }
      if (self) {
#pragma unroll
        for (int u = 0; u < GS_EPT; ++u) {
          ds_mac(sh, sl, wv[u].x, wv[u].y, wv[u].x, wv[u].y);
          ds_mac(sh, sl, wv[u].z, wv[u].w, wv[u].z, wv[u].w);
        }
        ds_renorm(sh, sl);
      }
#pragma unroll
      for (int k = 0; k < KM; ++k) {
        if (k >= nk0) break;
        const float4 *tv = gs_acquire(g, it, ok, status);
        float4 vv[GS_EPT];
#pragma unroll
        for (int u = 0; u < GS_EPT; ++u) {
          const int e = u * GS_CONS + tid;
          vv[u] = e < cnt ? tv[e] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < GS_EPT; ++u) {
          const float4 a = vv[u], b = wv[u];
          ds_mac(acc[k][0], acc[k][1], a.x, a.y, b.x, b.y);     // re += ar br
          ds_mac(acc[k][0], acc[k][1], a.z, a.w, b.z, b.w);     // re += ai bi
          ds_mac(acc[k][2], acc[k][3], a.x, a.y, b.z, b.w);     // im += ar bi
          ds_mac(acc[k][2], acc[k][3], -a.z, -a.w, b.x, b.y);   // im -= ai br
        }
        gs_release(g, it);   // after the tile's values are used
        ++it;
        ds_renorm(acc[k][0], acc[k][1]);
        ds_renorm(acc[k][2], acc[k][3]);
      }
    }
    // item epilogue: warp sums, then the eight warps combined in a fixed order
    const int nk = nk0 + (self ? 1 : 0);
#pragma unroll
    for (int k = 0; k <= KM; ++k) {
      if (k >= nk) break;
      const int kk = k < KM ? k : KM - 1;   // (k == KM only for the self entry)
      float4 t = k < nk0 ? make_float4(acc[kk][0], acc[kk][1], acc[kk][2], acc[kk][3])
                         : make_float4(sh, sl, 0.f, 0.f);   // entry nk0: ||w||^2
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float a = __shfl_xor_sync(0xffffffffu, t.x, o), b = __shfl_xor_sync(0xffffffffu, t.y, o);
        const float c = __shfl_xor_sync(0xffffffffu, t.z, o), d = __shfl_xor_sync(0xffffffffu, t.w, o);
        ds_add(t.x, t.y, a, b);
        ds_add(t.z, t.w, c, d);
      }
      if (lane == 0) red[warp][k] = t;
    }
    gs_consumer_sync();
    if (tid < nk) {
      float4 t = red[0][tid];
      for (int w8 = 1; w8 < GS_CONS / 32; ++w8) {
        const float4 o = red[w8][tid];
        ds_add(t.x, t.y, o.x, o.y);
        ds_add(t.z, t.w, o.z, o.w);
      }
      partial_all[(int64_t)r * ldp + (int64_t)tid * S + seg] = make_double2(ds_to_d(t.x, t.y), ds_to_d(t.z, t.w));
    }
    gs_consumer_sync();   // red is reused by the next item
  }
}

// ------------------------------------------------------------------ update
// Tiles per chunk: V_0 .. V_{nk-1}, then base.  Consumer thread t accumulates
// sum_k V_k c_k for entries t + 256 u of the chunk, then forms y from the base tile.
// base and y may be the same vector (the second pass updates in place): each chunk's
// base tile has landed in shared memory before any of its entries is written.
constexpr size_t gs_coef_offset() { return (gs_ring_bytes() + 15) & ~(size_t)15; }

template <bool NORM>
__global__ void __launch_bounds__(GS_THREADS, GS_CTAS_PER_SM)
k_gs_update(const float4 *__restrict__ V, int64_t ldv, int64_t ldvr, int nk, const double2 *__restrict__ coef_all,
            int ldc, const double *__restrict__ sc_all, const double2 *base_all, double2 *y_all, int64_t ldy,
            float4 *__restrict__ vout_all, int64_t n, int B, double2 *__restrict__ normpart_all, int S, int64_t ldp,
            const int *__restrict__ skip, const int *__restrict__ live, int scale, int32_t *status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double nsm[GS_CONS / 32];
  __shared__ double gsm;
  const GsRing g = gs_ring(smem_raw);
  float4 *csm = reinterpret_cast<float4 *>(smem_raw + gs_coef_offset());   // [nk] coefficients as float pairs
  gs_init(g);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int T = B * S;
  if (warp == GS_CONS / 32) {
    if (lane == 0)
      gs_produce(g, n, S, T, nk + 1, skip, live, status, [&](int r, int t) -> const char * {
        return t < nk ? reinterpret_cast<const char *>(V + (int64_t)r * ldvr + (int64_t)t * ldv)
                      : reinterpret_cast<const char *>(base_all + (int64_t)r * ldy);
      });
    return;
  }
  uint32_t it = 0;
  bool ok = true;
  int cur = -1;
  float2 gds = make_float2(1.f, 0.f);
  for (int q = blockIdx.x; q < T; q += gridDim.x) {
    const int r = q / S, seg = q - r * S;
    if (gs_item_off(r, skip, live)) continue;
    if (r != cur) {
      // this right-hand side's output scale g (one FP64 square root and division) and
      // projection coefficients coef_k sc_k^2 g as float pairs
      gs_consumer_sync();   // the previous right-hand side's coefficients are no longer read
      const double2 *coef = coef_all + (int64_t)r * ldc;
      const double *sc = sc_all + (int64_t)r * ldc;
      if (tid == 0) gsm = scale ? lazy_gamma(coef[nk].x) : 1.0;
      gs_consumer_sync();
      const double gg = gsm;
      gds = ds_split(gg);
      for (int k = tid; k < nk; k += GS_CONS) {
        const double2 c0 = coef[k];
        const double s2 = sc[k] * sc[k] * gg;
        const float2 cr = ds_split(c0.x * s2), ci = ds_split(c0.y * s2);
        csm[k] = make_float4(cr.x, cr.y, ci.x, ci.y);
      }
      gs_consumer_sync();
      cur = r;
    }
    double2 *y = y_all + (int64_t)r * ldy;
    float4 *vout = vout_all + (int64_t)r * ldvr;
    const int64_t e0 = (int64_t)seg * GS_ITEM, e1 = min(n, e0 + GS_ITEM);
    float nh = 0.f, nl = 0.f;   // double-single |y|^2 of this thread's entries
    for (int64_t c0 = e0; c0 < e1; c0 += GS_TILE) {
      const int cnt = (int)min((int64_t)GS_TILE, e1 - c0);
      float rh[GS_EPT], rl[GS_EPT], ih[GS_EPT], il[GS_EPT];
#pragma unroll
      for (int u = 0; u < GS_EPT; ++u) { rh[u] = rl[u] = ih[u] = il[u] = 0.f; }
#pragma unroll 2
      for (int k = 0; k < nk; ++k) {
        const float4 c = csm[k];
        const float4 *tv = gs_acquire(g, it, ok, status);
        float4 a[GS_EPT];
#pragma unroll
        for (int u = 0; u < GS_EPT; ++u) {
          const int e = u * GS_CONS + tid;
          a[u] = e < cnt ? tv[e] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < GS_EPT; ++u) {
          ds_mac(rh[u], rl[u], a[u].x, a[u].y, c.x, c.y);      // re += ar cr
          ds_mac(rh[u], rl[u], -a[u].z, -a[u].w, c.z, c.w);    // re -= ai ci
          ds_mac(ih[u], il[u], a[u].x, a[u].y, c.z, c.w);      // im += ar ci
          ds_mac(ih[u], il[u], a[u].z, a[u].w, c.x, c.y);      // im += ai cr
        }
        gs_release(g, it);   // after the tile's values are used
        ++it;
        if ((k & 7) == 7) {
#pragma unroll
          for (int u = 0; u < GS_EPT; ++u) { ds_renorm(rh[u], rl[u]); ds_renorm(ih[u], il[u]); }
        }
      }
      double2 bv[GS_EPT];
      {
        const double2 *tb = reinterpret_cast<const double2 *>(gs_acquire(g, it, ok, status));
#pragma unroll
        for (int u = 0; u < GS_EPT; ++u) {
          const int e = u * GS_CONS + tid;
          bv[u] = e < cnt ? tb[e] : make_double2(0.0, 0.0);
        }
      }
#pragma unroll
      for (int u = 0; u < GS_EPT; ++u) {
        const int e = u * GS_CONS + tid;
        if (e < cnt) {
          // y = g base - acc in double-single (g base as a double-single product), then one
          // FP64 add per component for the FP64 copy
          const float2 br = ds_split(bv[u].x), bi = ds_split(bv[u].y);
          float oh = 0.f, ol = 0.f, qh = 0.f, ql = 0.f;
          ds_mac(oh, ol, gds.x, gds.y, br.x, br.y);
          ds_mac(qh, ql, gds.x, gds.y, bi.x, bi.y);
          ds_renorm(oh, ol);
          ds_renorm(qh, ql);
          ds_add(oh, ol, -rh[u], -rl[u]);
          ds_add(qh, ql, -ih[u], -il[u]);
          y[c0 + e] = make_double2(ds_to_d(oh, ol), ds_to_d(qh, ql));
          vout[c0 + e] = make_float4(oh, ol, qh, ql);
          if (NORM) {
            ds_mac(nh, nl, oh, ol, oh, ol);
            ds_mac(nh, nl, qh, ql, qh, ql);
          }
        }
      }
      gs_release(g, it);   // the base tile, after its values are used
      ++it;
      if (NORM) ds_renorm(nh, nl);
    }
    if (NORM) {
      double nrm = ds_to_d(nh, nl);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
      if (lane == 0) nsm[warp] = nrm;
      gs_consumer_sync();
      if (tid == 0) {
        double s = 0.0;
        for (int w8 = 0; w8 < GS_CONS / 32; ++w8) s += nsm[w8];
        normpart_all[(int64_t)r * ldp + seg] = make_double2(s, 0.0);
      }
      gs_consumer_sync();   // nsm is reused by the next item
    }
  }
}

// ------------------------------------------------------------------ launchers
static int gs_grid(int T) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, std::min(T, GS_CTAS_PER_SM * sms));
}

int gs_items(int64_t n) { return (int)((n + GS_ITEM - 1) / GS_ITEM); }

cudaError_t launch_gs_dots(const float4 *V, int64_t ldv, int64_t ldvr, int nk0, const double2 *w, int64_t ldw,
                           int64_t n, int B, double2 *partial, int64_t ldp, const int *skip, const int *live, int self,
                           int32_t *status, cudaStream_t st) {
  const int S = gs_items(n);
  const dim3 grid(gs_grid(B * S));
  const size_t smem = gs_ring_bytes();
  cudaError_t e;
  if (nk0 <= 4) {
    if ((e = allow_smem(k_gs_dots<4>, smem)) != cudaSuccess) return e;
    k_gs_dots<4><<<grid, GS_THREADS, smem, st>>>(V, ldv, ldvr, nk0, w, ldw, n, B, partial, S, ldp, skip, live, self,
                                                 status);
  } else if (nk0 <= 8) {
    if ((e = allow_smem(k_gs_dots<8>, smem)) != cudaSuccess) return e;
    k_gs_dots<8><<<grid, GS_THREADS, smem, st>>>(V, ldv, ldvr, nk0, w, ldw, n, B, partial, S, ldp, skip, live, self,
                                                 status);
  } else if (nk0 <= kGsDotsMax) {
    if ((e = allow_smem(k_gs_dots<kGsDotsMax>, smem)) != cudaSuccess) return e;
    k_gs_dots<kGsDotsMax><<<grid, GS_THREADS, smem, st>>>(V, ldv, ldvr, nk0, w, ldw, n, B, partial, S, ldp, skip,
                                                          live, self, status);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_gs_update(const float4 *V, int64_t ldv, int64_t ldvr, int nk, const double2 *coef, int ldc,
                             const double *sc, const double2 *base, double2 *y, int64_t ldy, float4 *vout, int64_t n,
                             int B, double2 *normpart, int64_t ldp, const int *skip, const int *live, int scale,
                             int32_t *status, cudaStream_t st) {
  const int S = gs_items(n);
  const dim3 grid(gs_grid(B * S));
  const size_t smem = gs_coef_offset() + sizeof(float4) * (size_t)std::max(nk, 1);
  cudaError_t e;
  if (normpart) {
    if ((e = allow_smem(k_gs_update<true>, smem)) != cudaSuccess) return e;
    k_gs_update<true><<<grid, GS_THREADS, smem, st>>>(V, ldv, ldvr, nk, coef, ldc, sc, base, y, ldy, vout, n, B,
                                                      normpart, S, ldp, skip, live, scale, status);
  } else {
    if ((e = allow_smem(k_gs_update<false>, smem)) != cudaSuccess) return e;
    k_gs_update<false><<<grid, GS_THREADS, smem, st>>>(V, ldv, ldvr, nk, coef, ldc, sc, base, y, ldy, vout, n, B,
                                                       nullptr, S, ldp, skip, live, scale, status);
  }
  return cudaGetLastError();
}

}  // namespace hd
