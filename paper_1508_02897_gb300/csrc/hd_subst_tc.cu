// Preconditioner application on the tensor cores (storage HD_TCORE), for many
// right-hand sides sharing one factorisation.
//
// Each step of the forward and back block substitutions of Eq. (pmlij) is
//     Y = S_j^{-1} V,   V, Y: m x NR complex (NR = 16 right-hand sides per CTA).
// With S = Sr + i Si and the 2NR x m real operands A1 = [Vr ; Vi], A2 = [-Vi ; Vr],
//     [Yr ; Yi]^T-free form:  Y^T = A1 Sr^T + A2 Si^T   (rows: Yr, then Yi),
// two real products accumulated into one FP32 tile in tensor memory: tcgen05.mma
// kind::tf32 with M = 64 (rows 0..31 used: the 16 real and 16 imaginary parts),
// N = m rounded up to 8 (every row of S_j^{-1} in one instruction) and K = 8.
// A tcgen05.mma costs about the same whatever its M and N (measured: ~150 cycles
// per instruction on this GPU), so the rows of S_j^{-1} go on the wide N side and
// a step takes 2 m/8 instructions.  The factor of a box row is stored in TF32
// (rounded to nearest) as chunks of 8 columns, each chunk the real then the
// imaginary plane, each plane [mp8/8 row groups][2 core matrices along K][8 rows]
// [4 columns] (mp8 = m rounded up to 8): the no-swizzle K-major operand layout, so
// a chunk goes from HBM to shared memory in one bulk copy and feeds the MMA as is.
// With M = 64 the accumulator row i lives in TMEM lane 32 (i / 16) + i % 16.
//
// Warp roles in a CTA (one box, one group of 16 right-hand sides):
//   warps 0-3  epilogue: warps 0 and 1 copy the accumulator (Yr, Yi for all rows)
//              from tensor memory into a shared row-major tile; then each thread
//              takes rows a, finishes the step (w_j, or x_j = w_j - y, to the staging
//              vector) and writes the next step's V (rho - L w, or U x) into A1, A2;
//   warp 4     producer: streams the chunks through an mbarrier ring with
//              cp.async.bulk, in use order across steps;
//   warp 5     allocates tensor memory and issues the MMAs (one thread), frees each
//              ring stage with tcgen05.commit, and signals the finished tile.
// Every wait is bounded (flag ST_TIMEOUT and unwind); tensor memory is released
// only after a final commit confirms that no MMA is in flight.
#include "hd_internal.cuh"

namespace hd {

constexpr int TC_NR = 16;                    // right-hand sides per CTA
constexpr int TC_EPI = 128;                  // epilogue threads (TMEM lanes 0..127)
constexpr int TC_THREADS = TC_EPI + 64;      // + producer warp + MMA warp
constexpr int TC_TMEM_COLS = 256;            // N = mp8 <= 256 accumulator columns
constexpr uint32_t kTcWaitLimit = 1u << 24;
constexpr uint32_t kBLbo = 144;              // A1/A2: bytes between core matrices along K (conflict-free writes)
constexpr int kYsLd = 33;                    // row stride (floats) of the shared accumulator copy

namespace {

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool tbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool tbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
  for (uint32_t it = 0; it < kTcWaitLimit; ++it) {
    if (tbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u && *abort_flag) return false;
  }
  return false;
}
__device__ __forceinline__ void tbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void tbar_expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(bar))
               : "memory");
}
// Shared-memory matrix descriptor: start, leading (K-direction) and stride
// (M/N-direction) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t mdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// 32 consecutive 32-bit accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace

// Shared memory: A1, A2 [144 * mp8max bytes each] | ring [NS][64 * mp8max] | Ys [mp8max][33] floats |
// full[NS] | empty[NS] | dfull | bready | fin | tmem address | abort flag.  The M = 64 reads
// of A2 run 144 * mp8max bytes past its end (rows 32..63, never used), into the ring and Ys.
size_t subst_tc_smem(int ns, int mp8max) {
  return 2 * (size_t)kBLbo * mp8max + (size_t)ns * 64 * mp8max + (size_t)kYsLd * 4 * mp8max +
         (2 * (size_t)ns + 3) * 8 + 16;
}

__global__ void __launch_bounds__(TC_THREADS, 2)
k_subst_tc(const SubDev *__restrict__ subs, const double2 *__restrict__ pool, const float *__restrict__ factor,
           const double2 *__restrict__ rg, int NX, int64_t vec_stride, float2 *__restrict__ staging, int64_t stg_stride,
           int nrhs, int NS, int mp8max, int32_t *status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const SubDev s = subs[blockIdx.y];
  const int m = s.ex, rows = s.ey, mp8 = (m + 7) & ~7;
  const int r0 = blockIdx.x * TC_NR;
  const size_t stage_bytes = (size_t)64 * mp8max;
  unsigned char *A1 = smem_raw;
  unsigned char *A2 = A1 + (size_t)kBLbo * mp8max;
  unsigned char *ring = A2 + (size_t)kBLbo * mp8max;
  float *Ys = reinterpret_cast<float *>(ring + (size_t)NS * stage_bytes);
  uint64_t *full = reinterpret_cast<uint64_t *>(Ys + (size_t)kYsLd * mp8max);
  uint64_t *empty = full + NS;
  uint64_t *dfull = empty + NS;
  uint64_t *bready = dfull + 1;
  uint64_t *fin = bready + 1;
  uint32_t *tholder = reinterpret_cast<uint32_t *>(fin + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tholder + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bsbo = kBLbo * (uint32_t)(mp8max / 4);   // A1/A2: bytes between 8-row groups

  if (tid == 0) {
    for (int q = 0; q < NS; ++q) {
      tbar_init(&full[q], 1);
      tbar_init(&empty[q], 1);
    }
    tbar_init(dfull, 1);
    tbar_init(bready, TC_EPI);
    tbar_init(fin, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tholder)),
                 "r"((uint32_t)TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tholder;

  const int nck = mp8 / 8;                 // chunks (MMA K steps) per block
  const int nsteps = 2 * rows - 1;
  const int64_t total = (int64_t)nsteps * nck;
  const int64_t slot_floats = 2 * (int64_t)mp8 * mp8;
  const float *Fs = factor + 2 * s.foff;
  const uint32_t chunk_bytes = (uint32_t)(64 * mp8);

  if (warp == 4) {
    // ---------------- producer: chunks of every block in use order
    if (lane == 0) {
      int64_t issued = 0;
      bool ok = true;
      for (int64_t it = 0; it < total && ok; ++it) {
        const int st = (int)(it / nck), c = (int)(it - (int64_t)st * nck);
        const int j = st < rows ? st : 2 * rows - 2 - st;
        const int slot = (int)(it % NS);
        const uint32_t ph = (uint32_t)((it / NS) & 1);
        if (!tbar_wait(&empty[slot], ph ^ 1u, abort_flag)) { ok = false; break; }
        tbar_expect(&full[slot], chunk_bytes);
        bulk_copy(ring + (size_t)slot * stage_bytes, Fs + j * slot_floats + (int64_t)c * 16 * mp8, chunk_bytes,
                  &full[slot]);
        issued = it + 1;
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(status, ST_TIMEOUT);
      }
      for (int64_t it = max((int64_t)0, issued - NS); it < issued; ++it)
        tbar_wait(&full[it % NS], (uint32_t)((it / NS) & 1), abort_flag);
    }
    return;
  }

  if (warp == 5) {
    // ---------------- MMA issuer (one thread); the warp owns the tensor memory
    if (lane == 0) {
      // D f32, A and B tf32, both K-major, N = mp8, M = 64
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(mp8 >> 3) << 17) | ((64u >> 4) << 24);
      const uint32_t a1 = su32(A1), a2 = su32(A2);
      int64_t it = 0;
      bool ok = true;
      for (int st = 0; st < nsteps && ok; ++st) {
        if (!tbar_wait(bready, (uint32_t)(st & 1), abort_flag)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int c = 0; c < nck; ++c, ++it) {
          const int slot = (int)(it % NS);
          if (!tbar_wait(&full[slot], (uint32_t)((it / NS) & 1), abort_flag)) { ok = false; break; }
          const uint32_t sb = su32(ring + (size_t)slot * stage_bytes);
          mma_tf32(tmem, mdesc(a1 + (uint32_t)c * 2 * kBLbo, kBLbo, bsbo), mdesc(sb, 128, 256), idesc, c > 0 ? 1u : 0u);
          mma_tf32(tmem, mdesc(a2 + (uint32_t)c * 2 * kBLbo, kBLbo, bsbo), mdesc(sb + (uint32_t)(32 * mp8), 128, 256),
                   idesc, 1u);
          mma_commit(&empty[slot]);   // the stage is free once these MMAs have read it
        }
        if (!ok) break;
        mma_commit(dfull);
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(status, ST_TIMEOUT);
      }
      mma_commit(fin);                          // arrives once every MMA issued above is done
      tbar_wait(fin, 0, abort_flag);
      tbar_wait(bready, (uint32_t)(nsteps & 1), abort_flag);   // epilogue done reading TMEM
    }
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TC_TMEM_COLS)
                 : "memory");
    return;
  }

  // ---------------- epilogue warps: thread e owns rows a = e and a = 128 + e
  const int e = tid;
  const double2 *a1c = pool + s.aoff;
  const double2 *a2c = a1c + 2 * m + 1;
  const double2 *ia2f = a2c + rows;
  // A1/A2 element (n, k) at (n/8)*bsbo + (k/4)*kBLbo + (n%8)*16 + (k%4)*4 bytes:
  // A1 = [Vr ; Vi], A2 = [-Vi ; Vr] (row n < 16: real parts, 16 <= n < 32: imaginary)
  auto put_v = [&](int a, int q, float2 v) {
    const uint32_t kofs = (uint32_t)(a >> 2) * kBLbo + (uint32_t)(a & 3) * 4;
    const float vr = tf32_rn(v.x), vi = tf32_rn(v.y);
    const int n1 = q, n2 = TC_NR + q;
    *reinterpret_cast<float *>(A1 + (n1 >> 3) * bsbo + kofs + (n1 & 7) * 16) = vr;
    *reinterpret_cast<float *>(A1 + (n2 >> 3) * bsbo + kofs + (n2 & 7) * 16) = vi;
    *reinterpret_cast<float *>(A2 + (n1 >> 3) * bsbo + kofs + (n1 & 7) * 16) = -vi;
    *reinterpret_cast<float *>(A2 + (n2 >> 3) * bsbo + kofs + (n2 & 7) * 16) = vr;
  };
  float2 a1[2];
  bool ownx[2];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int a = 128 * t + e;
    const double2 v = a < m ? a1c[a] : make_double2(0.0, 0.0);
    a1[t] = make_float2((float)v.x, (float)v.y);
    const int gx = s.ex0 + a;
    ownx[t] = a < m && gx >= s.ox0 && gx < s.ox1;
  }
  // V_0 = rho_0 (zero in the K padding rows m <= a < mp8)
  {
    const int gy = s.ey0;
    const bool owny = gy >= s.oy0 && gy < s.oy1;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int a = 128 * t + e;
      if (a >= mp8) continue;
      for (int q = 0; q < TC_NR; ++q) {
        float2 rho = make_float2(0.f, 0.f);
        if (owny && ownx[t] && r0 + q < nrhs) {
          const double2 rv = rg[(int64_t)(r0 + q) * vec_stride + (int64_t)gy * NX + s.ex0 + a];
          rho = make_float2((float)rv.x, (float)rv.y);
        }
        put_v(a, q, rho);
      }
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  tbar_arrive(bready);

  for (int st = 0; st < nsteps; ++st) {
    const bool fwd = st < rows;
    const int j = fwd ? st : 2 * rows - 2 - st;
    // the next step's coupling: forward rho_{j+1} - L_{j+1} w_j, backward U_{jn} x_{jn+1}
    const int sn = st + 1;
    const bool has_next = sn < nsteps;
    const bool nfwd = sn < rows;
    const int jn = nfwd ? sn : 2 * rows - 2 - sn;
    float2 cpl = make_float2(0.f, 0.f);
    bool owny_n = false;
    int gy_n = 0;
    if (has_next) {
      const double2 c = nfwd ? ia2f[jn] : ia2f[jn + 1];
      cpl = make_float2((float)c.x, (float)c.y);
      gy_n = s.ey0 + jn;
      owny_n = nfwd && gy_n >= s.oy0 && gy_n < s.oy1;
    }
    // operands that do not depend on this step's product, loaded while the MMAs run:
    // the staged w_j (backward) or the next row's residual (forward)
    float2 pre[2][TC_NR];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int a = 128 * t + e;
#pragma unroll
      for (int q = 0; q < TC_NR; ++q) {
        float2 v = make_float2(0.f, 0.f);
        const bool live = a < m && r0 + q < nrhs;
        if (live && !fwd) {
          v = staging[(int64_t)(r0 + q) * stg_stride + s.soff + (int64_t)j * m + a];
        } else if (live && has_next && nfwd && owny_n && ownx[t]) {
          const double2 rv = rg[(int64_t)(r0 + q) * vec_stride + (int64_t)gy_n * NX + s.ex0 + a];
          v = make_float2((float)rv.x, (float)rv.y);
        }
        pre[t][q] = v;
      }
    }
    // a timed-out wait must not split the epilogue warps around the named barrier:
    // every thread reaches it, and all of them leave together if anyone gave up
    const bool got = __all_sync(0xffffffffu, tbar_wait(dfull, (uint32_t)(st & 1), abort_flag));
    if (!got && lane == 0) {
      *abort_flag = 1;
      atomicOr(status, ST_TIMEOUT);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // accumulator rows 0..15 (Yr) sit in TMEM lanes 0..15, rows 16..31 (Yi) in lanes 32..47:
    // warps 0 and 1 copy them, 32 columns (rows a of the box) at a time, into Ys[a][n]
    if (warp < 2 && got) {
      const int n = 16 * warp + lane;
      for (int c0 = 0; c0 < mp8; c0 += 32) {
        float y[32];
        tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, y);   // warp-collective
        if (lane < 16)
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (c0 + i < mp8) Ys[(c0 + i) * kYsLd + n] = y[i];
      }
    }
    // barrier of the epilogue warps only, OR-reducing "give up" so that all leave together
    uint32_t quit;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(quit)
        : "r"((!got || *abort_flag) ? 1u : 0u), "r"(TC_EPI)
        : "memory");
    if (quit) break;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int a = 128 * t + e;
      if (a >= m) break;
      const float2 lc = cmul(a1[t], cpl);   // L_{jn} or U_{jn} entry of row a
#pragma unroll
      for (int q = 0; q < TC_NR; ++q) {
        const float2 yq = make_float2(Ys[a * kYsLd + q], Ys[a * kYsLd + TC_NR + q]);
        const float2 out = fwd ? yq : csub(pre[t][q], yq);
        if (r0 + q < nrhs) staging[(int64_t)(r0 + q) * stg_stride + s.soff + (int64_t)j * m + a] = out;
        if (has_next) put_v(a, q, nfwd ? cfms(lc, out, fwd ? pre[t][q] : make_float2(0.f, 0.f)) : cmul(lc, out));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    tbar_arrive(bready);
  }
}

// Stages of the ring: as many as fit beside the B operands for the CTAs that
// share an SM (one or two).
cudaError_t launch_subst_tc(hd_ctx *ctx, const double2 *r, int nrhs, int64_t vec_stride, void *staging,
                            int64_t stg_stride, cudaStream_t st) {
  const int mp8max = (ctx->max_m + 7) & ~7;
  if (mp8max > 256) return cudaErrorInvalidValue;
  const int groups = (nrhs + TC_NR - 1) / TC_NR;
  int dev = 0, sms = 152, optin = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
#ifndef TC_CTAS_PER_SM
#define TC_CTAS_PER_SM 2
#endif
  const int per_sm = ((int64_t)ctx->nsub * groups > sms) ? TC_CTAS_PER_SM : 1;
  const size_t budget = std::min((size_t)optin, (size_t)(per_sm == 2 ? 110 : 220) * 1024);
  int ns = 2;
  while (ns < 16 && subst_tc_smem(ns + 1, mp8max) <= budget) ++ns;
  const size_t smem = subst_tc_smem(ns, mp8max);
  cudaError_t e = allow_smem(k_subst_tc, smem);
  if (e != cudaSuccess) return e;
  // the groups of one box are neighbours in launch order: they run together and read
  // the box's factor chunks at about the same time, so L2 serves most repeated reads
  dim3 grid(groups, ctx->nsub);
  k_subst_tc<<<grid, TC_THREADS, smem, st>>>(ctx->d_subs, ctx->d_lpool, reinterpret_cast<const float *>(ctx->factor), r,
                                             ctx->NX, vec_stride, reinterpret_cast<float2 *>(staging), stg_stride,
                                             nrhs, ns, mp8max, ctx->d_status);
  return cudaGetLastError();
}

}  // namespace hd
