// Preconditioner application, Eq. (ddm0) + Eq. (pc):
//   z = sum_ij E_ij^T A_ij^{-1} X_ij r.
//
// k_subst (one CTA per box) fuses the restriction X_ij r (a gather of the
// owned part of each grid row of the box straight from the global residual)
// with the forward block substitution
//     w_0 = S_0^{-1} rho_0,   w_j = S_j^{-1} (rho_j - L_j w_{j-1}),
// and the back substitution
//     x_last = w_last,        x_j = w_j - S_j^{-1} (U_j x_{j+1}),
// leaving the local solution over the whole box (PML area included) in the
// staging buffer.  Each step is one m x m complex GEMV against a stored
// S_j^{-1}, so the kernel streams 2 rows - 1 dense m x m blocks per box: it is
// HBM-bound.  The stream of factor blocks does not depend on the vectors, so a
// producer warp copies them ahead with bulk asynchronous copies
// (cp.async.bulk, completion counted on an mbarrier) into a ring of NS shared
// memory stages of CH columns each, across step boundaries; the consumer
// warps accumulate y[a] = sum_b S[a][b] v[b] from shared memory (thread t owns
// outputs a = t + CT*e) and release each stage on its "empty" mbarrier.
// Every wait is bounded: on timeout the kernel flags ST_TIMEOUT, stops issuing
// copies, lets every warp run to the end, and the producer waits for its own
// copies still in flight before the CTA exits.
//
// k_gather then forms z cell by cell as a fixed-order sum over the (at most
// 3 x 3, in practice 2 x 2) boxes whose extent covers the cell: deterministic,
// no atomics.
#include "hd_internal.cuh"

namespace hd {

constexpr uint32_t kWaitLimit = 1u << 24;   // try_wait rounds before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; false on timeout or when another warp already gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && *abort_flag) return false;
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void consumer_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

template <typename T> __host__ __device__ constexpr int chunk_cols() { return sizeof(T) == 8 ? 4 : 2; }

// Shared memory layout: ring [NS][CH*ldmax] | vs [NR][ldmax] | full[NS] | empty[NS] | abort
template <typename T>
__host__ __device__ inline size_t subst_smem(int ns, int ldmax, int nr) {
  size_t stage = (size_t)chunk_cols<T>() * ldmax * sizeof(T);
  size_t o = (size_t)ns * stage + (size_t)nr * ldmax * sizeof(T);
  o = (o + 15) & ~(size_t)15;
  return o + 2 * (size_t)ns * sizeof(uint64_t) + 16;
}

// One CTA per (box, group of NR right-hand sides): every factor block is read
// once per group and applied to NR vectors.
template <typename R, int CT, int NA, int NR>
__global__ void __launch_bounds__(CT + 32)
k_subst(const SubDev *__restrict__ subs, const double2 *__restrict__ pool, const C<R> *__restrict__ factor,
        const double2 *__restrict__ rg, int NX, int64_t vec_stride, C<R> *__restrict__ staging, int64_t stg_stride,
        int nrhs, int NS, int ldmax, int32_t *status) {
  using T = C<R>;
  constexpr int CH = chunk_cols<T>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const SubDev s = subs[blockIdx.x];
  const int m = s.ex, rows = s.ey, ldm = s.ldm;
  const int r0 = blockIdx.y * NR;
  const size_t stage_elems = (size_t)CH * ldmax;
  T *ring = reinterpret_cast<T *>(smem_raw);
  T *vs = ring + (size_t)NS * stage_elems;     // [NR][ldmax]
  size_t off = ((size_t)NS * stage_elems + (size_t)NR * ldmax) * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + off);
  uint64_t *empty = full + NS;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + NS);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    for (int q = 0; q < NS; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], CT / 32);
    }
    *abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();

  const int nck = (m + CH - 1) / CH;             // chunks per factor block
  const int64_t total = (int64_t)(2 * rows - 1) * nck;
  const int64_t slot_elems = (int64_t)m * ldm;
  const T *Fs = factor + s.foff;

  if (warp == CT / 32) {
    // ---------------- producer warp: stream the factor blocks in use order
    if (lane == 0) {
      int64_t issued = 0;
      bool ok = true;
      for (int64_t it = 0; it < total && ok; ++it) {
        const int st = (int)(it / nck), c = (int)(it - (int64_t)st * nck);
        const int j = st < rows ? st : 2 * rows - 2 - st;
        const int slot = (int)(it % NS);
        const uint32_t ph = (uint32_t)((it / NS) & 1);
        if (!mbar_wait(&empty[slot], ph ^ 1u, abort_flag)) { ok = false; break; }
        const int cols = min(CH, m - c * CH);
        const uint32_t bytes = (uint32_t)(cols * ldm * sizeof(T));
        mbar_arrive_expect_tx(&full[slot], bytes);
        bulk_g2s(ring + (size_t)slot * stage_elems, Fs + j * slot_elems + (int64_t)c * CH * ldm, bytes, &full[slot]);
        issued = it + 1;
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(status, ST_TIMEOUT);
      }
      // no copy may still be landing in shared memory when the CTA exits
      for (int64_t it = max((int64_t)0, issued - NS); it < issued; ++it)
        mbar_wait(&full[it % NS], (uint32_t)((it / NS) & 1), abort_flag);
    }
    return;
  }

  // ---------------- consumer warps
  const double2 *a1c = pool + s.aoff;
  const double2 *a2c = a1c + 2 * m + 1;
  const double2 *ia2f = a2c + rows;
  T a1[NA], w[NA][NR];
  bool ownx[NA];
#pragma unroll
  for (int e = 0; e < NA; ++e) {
    const int a = tid + CT * e;
    const int gx = s.ex0 + a;
    ownx[e] = a < m && gx >= s.ox0 && gx < s.ox1;
    const double2 t = a < m ? a1c[a] : make_double2(0, 0);
    a1[e] = mk<T>((R)t.x, (R)t.y);
#pragma unroll
    for (int q = 0; q < NR; ++q) w[e][q] = mk<T>(0, 0);
  }
  int64_t it = 0;
  bool ok = true;
  for (int st = 0; st < 2 * rows - 1; ++st) {
    const bool fwd = st < rows;
    const int j = fwd ? st : 2 * rows - 2 - st;
    consumer_sync(CT);   // the previous step's reads of vs are done
    if (fwd) {
      const int gy = s.ey0 + j;
      const bool owny = gy >= s.oy0 && gy < s.oy1;
      const double2 isd = ia2f[j];
      const T is = mk<T>((R)isd.x, (R)isd.y);
#pragma unroll
      for (int e = 0; e < NA; ++e) {
        const int a = tid + CT * e;
        if (a < m) {
          const T la = cmul(a1[e], is);
#pragma unroll
          for (int q = 0; q < NR; ++q) {
            T rho = mk<T>(0, 0);
            if (owny && ownx[e] && r0 + q < nrhs) {
              const double2 rv = rg[(int64_t)(r0 + q) * vec_stride + (int64_t)gy * NX + s.ex0 + a];
              rho = mk<T>((R)rv.x, (R)rv.y);
            }
            vs[q * ldmax + a] = j > 0 ? cfms(la, w[e][q], rho) : rho;   // rho_j - L_j w_{j-1}
          }
        }
      }
    } else {
      const double2 ind = ia2f[j + 1];
      const T in = mk<T>((R)ind.x, (R)ind.y);
#pragma unroll
      for (int e = 0; e < NA; ++e) {
        const int a = tid + CT * e;
        if (a < m) {
          const T ua = cmul(a1[e], in);
#pragma unroll
          for (int q = 0; q < NR; ++q) vs[q * ldmax + a] = cmul(ua, w[e][q]);   // U_j x_{j+1}
        }
      }
    }
    consumer_sync(CT);
    T acc[NA][NR];
#pragma unroll
    for (int e = 0; e < NA; ++e)
#pragma unroll
      for (int q = 0; q < NR; ++q) acc[e][q] = mk<T>(0, 0);
    for (int c = 0; c < nck; ++c, ++it) {
      const int slot = (int)(it % NS);
      if (ok && !mbar_wait(&full[slot], (uint32_t)((it / NS) & 1), abort_flag)) {
        ok = false;
        *abort_flag = 1;
        atomicOr(status, ST_TIMEOUT);
      }
      const T *blk = ring + (size_t)slot * stage_elems;
      const int b0 = c * CH;
      const int cols = min(CH, m - b0);
#pragma unroll
      for (int b = 0; b < CH; ++b) {
        if (b < cols) {
          T sv[NA];
#pragma unroll
          for (int e = 0; e < NA; ++e) {
            const int a = tid + CT * e;
            sv[e] = a < m ? blk[b * ldm + a] : mk<T>(0, 0);
          }
#pragma unroll
          for (int q = 0; q < NR; ++q) {
            const T vb = vs[q * ldmax + b0 + b];
#pragma unroll
            for (int e = 0; e < NA; ++e) acc[e][q] = cfma(sv[e], vb, acc[e][q]);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot]);
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      if (r0 + q >= nrhs) continue;
      T *stg = staging + (int64_t)(r0 + q) * stg_stride + s.soff;
#pragma unroll
      for (int e = 0; e < NA; ++e) {
        const int a = tid + CT * e;
        if (a < m) {
          if (fwd) {
            w[e][q] = acc[e][q];
            stg[(int64_t)j * m + a] = acc[e][q];
          } else {
            const T x = csub(stg[(int64_t)j * m + a], acc[e][q]);
            w[e][q] = x;
            stg[(int64_t)j * m + a] = x;
          }
        }
      }
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(256)
k_gather(const SubDev *__restrict__ subs, const AxisDev *__restrict__ axx, const AxisDev *__restrict__ axy,
         const int32_t *__restrict__ nearx, const int32_t *__restrict__ neary, int nbx, int nby,
         const C<R> *__restrict__ staging_all, int64_t stg_stride, double2 *__restrict__ z_all, int64_t vec_stride,
         int NX) {
  int gx = blockIdx.x * blockDim.x + threadIdx.x;
  int gy = blockIdx.y;
  const C<R> *staging = staging_all + (int64_t)blockIdx.z * stg_stride;
  double2 *z = z_all + (int64_t)blockIdx.z * vec_stride;
  if (gx >= NX) return;
  const int ix = nearx[gx], iy = neary[gy];
  double2 acc = make_double2(0.0, 0.0);
  for (int jy = max(iy - 1, 0); jy <= min(iy + 1, nby - 1); ++jy) {
    const AxisDev ay = axy[jy];
    if (gy < ay.e0 || gy >= ay.e1) continue;
    for (int jx = max(ix - 1, 0); jx <= min(ix + 1, nbx - 1); ++jx) {
      const AxisDev ax = axx[jx];
      if (gx < ax.e0 || gx >= ax.e1) continue;
      const int64_t base = subs[jy * nbx + jx].soff;
      const int ex = ax.e1 - ax.e0;
      const C<R> v = staging[base + (int64_t)(gy - ay.e0) * ex + (gx - ax.e0)];
      acc.x += (double)v.x;
      acc.y += (double)v.y;
    }
  }
  z[(int64_t)gy * NX + gx] = acc;
}

// Ring depth: as deep as shared memory allows for the CTAs that share an SM.
template <typename T>
static int ring_stages(const hd_ctx *ctx, int ldmax, int nr, int groups) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ctas = (int64_t)ctx->nsub * groups;
  const int per_sm = (int)std::min<int64_t>(7, (ctas + sms - 1) / sms);
  const size_t budget = (size_t)200 * 1024 / (size_t)std::max(1, per_sm);
  const size_t stage = (size_t)chunk_cols<T>() * ldmax * sizeof(T);
  const size_t fixed = (size_t)nr * ldmax * sizeof(T) + 64;
  int ns = budget > fixed ? (int)((budget - fixed) / stage) : 2;
  return std::min(32, std::max(2, ns));
}

// Right-hand sides per CTA: one factor read serves NR vectors.
static int rhs_per_cta(int nrhs) { return nrhs >= 8 ? 8 : (nrhs >= 4 ? 4 : (nrhs >= 2 ? 2 : 1)); }

size_t subst_ring_bytes(const hd_ctx *ctx, int *stages) {
  const int ldmax = (ctx->max_m + 1) & ~1;
  if (ctx->prec == HD_C64) {
    int ns = ring_stages<float2>(ctx, ldmax, 1, 1);
    if (stages) *stages = ns;
    return subst_smem<float2>(ns, ldmax, 1);
  }
  int ns = ring_stages<double2>(ctx, ldmax, 1, 1);
  if (stages) *stages = ns;
  return subst_smem<double2>(ns, ldmax, 1);
}

template <typename R, int CT, int NR>
static cudaError_t launch_subst(hd_ctx *ctx, const double2 *r, int nrhs, int64_t vec_stride, void *staging,
                                int64_t stg_stride, cudaStream_t st) {
  using T = C<R>;
  const int ldmax = (ctx->max_m + 1) & ~1;
  const int groups = (nrhs + NR - 1) / NR;
  const int ns = ring_stages<T>(ctx, ldmax, NR, groups);
  const size_t smem = subst_smem<T>(ns, ldmax, NR);
  cudaError_t e = cudaFuncSetAttribute(k_subst<R, CT, 2, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(ctx->nsub, groups);
  k_subst<R, CT, 2, NR><<<grid, CT + 32, smem, st>>>(ctx->d_subs, ctx->d_lpool,
                                                     reinterpret_cast<const T *>(ctx->factor), r, ctx->NX, vec_stride,
                                                     reinterpret_cast<T *>(staging), stg_stride, nrhs, ns, ldmax,
                                                     ctx->d_status);
  return cudaGetLastError();
}

template <typename R, int CT>
static cudaError_t launch_subst_nr(hd_ctx *ctx, const double2 *r, int nrhs, int64_t vs, void *stg, int64_t ss,
                                   cudaStream_t st) {
  switch (rhs_per_cta(nrhs)) {
    case 8: return launch_subst<R, CT, 8>(ctx, r, nrhs, vs, stg, ss, st);
    case 4: return launch_subst<R, CT, 4>(ctx, r, nrhs, vs, stg, ss, st);
    case 2: return launch_subst<R, CT, 2>(ctx, r, nrhs, vs, stg, ss, st);
    default: return launch_subst<R, CT, 1>(ctx, r, nrhs, vs, stg, ss, st);
  }
}

template <typename R>
static cudaError_t launch_apply_r(hd_ctx *ctx, const double2 *r, int64_t rs, double2 *z, int64_t zs, int nrhs,
                                  void *staging, cudaStream_t st) {
  tic(ctx, T_SUBST, st);
  cudaError_t e = ctx->max_m <= 192 ? launch_subst_nr<R, 96>(ctx, r, nrhs, rs, staging, ctx->staging_elems, st)
                                    : launch_subst_nr<R, 128>(ctx, r, nrhs, rs, staging, ctx->staging_elems, st);
  toc(ctx, T_SUBST, st, 1);
  if (e != cudaSuccess) return e;
  dim3 grid((ctx->NX + 255) / 256, ctx->NY, nrhs);
  tic(ctx, T_GATHER, st);
  k_gather<R><<<grid, 256, 0, st>>>(ctx->d_subs, ctx->d_axx, ctx->d_axy, ctx->d_nearx, ctx->d_neary, ctx->nbx,
                                    ctx->nby, reinterpret_cast<const C<R> *>(staging), ctx->staging_elems, z, zs,
                                    ctx->NX);
  toc(ctx, T_GATHER, st, 1);
  return cudaGetLastError();
}

int run_apply(hd_ctx *ctx, const double2 *r, int64_t rs, double2 *z, int64_t zs, int nrhs, void *staging,
              cudaStream_t st) {
  cudaError_t e = ctx->prec == HD_C64 ? launch_apply_r<float>(ctx, r, rs, z, zs, nrhs, staging, st)
                                      : launch_apply_r<double>(ctx, r, rs, z, zs, nrhs, staging, st);
  if (e != cudaSuccess) return cuda_fail(e, "preconditioner launch");
  return HD_OK;
}

}  // namespace hd
