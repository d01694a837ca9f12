// Preconditioner application on the tensor cores with FP32-grade products (storage
// HD_TCORE | HD_TF32X3), for many right-hand sides sharing one factorisation.
//
// The steps are those of the forward and back block substitutions of Eq. (pmlij),
//     Y = S_j^{-1} V,   V, Y: m x 32 complex (32 right-hand sides per CTA),
// but every operand is carried as a pair of TF32 numbers x = x_hi + x_lo (x_hi = x
// rounded to TF32, x_lo = the remainder rounded to TF32, |x - x_hi - x_lo| <= 2^-22 |x|)
// and every product takes the partial products hi*hi + lo*hi + hi*lo (+ lo*lo, which
// comes along), accumulated in FP32 ("3xTF32").  The relative error of a product is then
// of the order of FP32's, against TF32's 2^-11 for the single-plane storage.
//
// MMA shape: tcgen05.mma kind::tf32, M = 128, N = m rounded up to 16, K = 8.  The 128
// rows of the A operands hold, for the warp quarter w (right-hand sides 8w .. 8w+7), the
// rows [Vr_hi; Vr_lo; Vi_hi; Vi_lo] (8 each) in A1 and [-Vi_hi; -Vi_lo; Vr_hi; Vr_lo]
// in A2.  Per 8-column chunk of S_j^{-1}:
//     D += A1 Sr_hi^T + A2 Si_hi^T + A1 Sr_lo^T + A2 Si_lo^T,
// so accumulator row (w, part, s) is the hi or lo part of Yr (parts 0, 1) or Yi (parts
// 2, 3) of right-hand side 8w + s, and the epilogue adds the parts with two lane
// exchanges.  Four MMAs per chunk serve 32 right-hand sides: the instruction count per
// right-hand side of the TF32 path (two MMAs per chunk for 16), and the same factor bytes
// per right-hand side (16 bytes per entry, read once per 32).
//
// Pipelining inside the CTA: two accumulators in tensor memory (even and odd steps).
// The epilogue of step t reads its accumulator 32 columns (rows a of the box) at a time,
// writes those rows of the output and the same 32 columns of the next step's V into
// A1/A2 (the next step's K range), and arrives on that column group's mbarrier; the MMAs
// of step t + 1 start on a column group as soon as it is complete, into the other
// accumulator, so the tensor cores work while the epilogue runs.  Each epilogue thread
// issues the global loads of the operands of its whole step that do not depend on the
// product (the staged w_j of a backward step, the next grid row's residual of a forward
// step) before it waits for the accumulator.
//
// Warp roles: warps 0-3 epilogue (thread = tensor-memory lane), warp 4 producer (factor
// chunks through an mbarrier ring with cp.async.bulk, in use order across steps, after
// asking L2 for them a few chunks ahead: the ring holds two to four chunks beside the A
// operands, too few to cover HBM's latency on its own), warp 5
// tensor-memory owner and MMA issuer (one thread).  Every wait is bounded (flag
// ST_TIMEOUT and unwind); tensor memory is released only after a final commit confirms
// that no MMA is in flight and the epilogue has finished reading it.
#include "hd_internal.cuh"
#include "hd_tc.cuh"

namespace hd {

namespace {

constexpr int X3_NR = 32;                     // right-hand sides per CTA
constexpr int X3_EPI = 128;                   // epilogue threads (tensor-memory lanes 0..127)
constexpr int X3_THREADS = X3_EPI + 64;       // + producer warp + MMA warp
constexpr int X3_TMEM_COLS = 512;             // two accumulators of up to 256 columns
constexpr uint32_t X3_HALF = 256;             // column offset of the odd-step accumulator
constexpr uint32_t kX3Lbo = 128;              // A1/A2: bytes between core matrices along K
constexpr int X3_GROUPS = (kMaxBoxWidthX3 + 31) / 32;   // 32-column groups of the widest box
constexpr size_t kX3Tail = 256;               // the last plane's N padding (m rounded to 16) reads past the ring
constexpr int kX3Prefetch = 8;                // chunks the producer asks L2 for ahead of its copies

__device__ __forceinline__ void bar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::su32(bar)) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc::su32(dst)),
               "l"(src), "r"(bytes), "r"(tc::su32(bar))
               : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// 32 consecutive 32-bit accumulator columns of this thread's lane (warp-collective, waits).
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
__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Writes columns k0 .. k0+7 of right-hand side s (warp quarter w) into A1 and A2: the
// four part rows of each, two 16-byte stores per row.  A1/A2 element (n, k) sits at
// (n / 8) * sbo + (k / 4) * kX3Lbo + (n % 8) * 16 + (k % 4) * 4 bytes.
__device__ __forceinline__ void put_v8(unsigned char *A1, unsigned char *A2, uint32_t sbo, int w, int s, int k0,
                                       const float2 *v) {
  float rh[8], rl[8], ih[8], il[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    rh[i] = tf32_rn(v[i].x);
    rl[i] = tf32_rn(v[i].x - rh[i]);
    ih[i] = tf32_rn(v[i].y);
    il[i] = tf32_rn(v[i].y - ih[i]);
  }
  const uint32_t base = (uint32_t)(k0 >> 2) * kX3Lbo + (uint32_t)s * 16;
  auto row = [&](unsigned char *A, int part) -> float4 * {
    return reinterpret_cast<float4 *>(A + (size_t)(4 * w + part) * sbo + base);
  };
  auto st2 = [&](float4 *p, const float *x, float sg) {
    p[0] = make_float4(sg * x[0], sg * x[1], sg * x[2], sg * x[3]);
    p[kX3Lbo / 16] = make_float4(sg * x[4], sg * x[5], sg * x[6], sg * x[7]);
  };
  st2(row(A1, 0), rh, 1.f);
  st2(row(A1, 1), rl, 1.f);
  st2(row(A1, 2), ih, 1.f);
  st2(row(A1, 3), il, 1.f);
  st2(row(A2, 0), ih, -1.f);
  st2(row(A2, 1), il, -1.f);
  st2(row(A2, 2), rh, 1.f);
  st2(row(A2, 3), rl, 1.f);
}

}  // namespace

// Shared memory: A1, A2 [16 row groups][mp8max / 4 core matrices][128 B] | ring [NS][128 mp8max]
// | tail padding | lA [mp8max] float2 | full[NS] | empty[NS] | dfull | aready[X3_GROUPS] | edone
// | fin | tensor-memory address | abort flag.
static size_t subst_x3_smem(int ns, int mp8max) {
  return 2 * (size_t)512 * mp8max + (size_t)ns * 128 * mp8max + kX3Tail + 8 * (size_t)mp8max +
         (2 * (size_t)ns + 3 + X3_GROUPS) * 8 + 16;
}

__global__ void __launch_bounds__(X3_THREADS, 1)
k_subst_x3(const SubDev *__restrict__ subs, const double2 *__restrict__ pool, const float *__restrict__ factor,
           const double2 *__restrict__ rg, int NX, int64_t vec_stride, float2 *__restrict__ staging, int64_t stg_stride,
           int nrhs, int NS, int mp8max, int32_t *status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const SubDev s = subs[blockIdx.y];
  const int m = s.ex, rows = s.ey, mp8 = (m + 7) & ~7, mp16 = (m + 15) & ~15;
  const int r0 = blockIdx.x * X3_NR;
  const size_t stage_bytes = (size_t)128 * mp8max;
  const uint32_t asbo = kX3Lbo * (uint32_t)(mp8max / 4);   // A1/A2: bytes between 8-row groups
  unsigned char *A1 = smem_raw;
  unsigned char *A2 = A1 + (size_t)16 * asbo;
  unsigned char *ring = A2 + (size_t)16 * asbo;
  float2 *lA = reinterpret_cast<float2 *>(ring + (size_t)NS * stage_bytes + kX3Tail);
  uint64_t *full = reinterpret_cast<uint64_t *>(lA + mp8max);
  uint64_t *empty = full + NS;
  uint64_t *dfull = empty + NS;
  uint64_t *aready = dfull + 1;
  uint64_t *edone = aready + X3_GROUPS;
  uint64_t *fin = edone + 1;
  uint32_t *tholder = reinterpret_cast<uint32_t *>(fin + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tholder + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ngrp = (mp8 + 31) / 32;

  if (tid == 0) {
    for (int q = 0; q < NS; ++q) {
      tc::bar_init(&full[q], 1);
      tc::bar_init(&empty[q], 1);
    }
    tc::bar_init(dfull, 1);
    for (int g = 0; g < X3_GROUPS; ++g) tc::bar_init(&aready[g], X3_EPI);
    tc::bar_init(edone, X3_EPI);
    tc::bar_init(fin, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {  // the sub-diagonal band entries of the box's rows (the coupling L / U of Eq. (pmlij)), zero past m
    const double2 *a1c = pool + s.aoff;
    for (int a = tid; a < mp8max; a += X3_THREADS) {
      const double2 v = a < m ? a1c[a] : make_double2(0.0, 0.0);
      lA[a] = make_float2((float)v.x, (float)v.y);
    }
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::su32(tholder)),
                 "r"((uint32_t)X3_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tholder;

  const int nck = mp8 / 8;                 // chunks (MMA K steps) per block
  const int nsteps = 2 * rows - 1;
  const int64_t total = (int64_t)nsteps * nck;
  const int64_t slot_floats = 4 * (int64_t)mp8 * mp8;
  const float *Fs = factor + 2 * s.foff;
  const uint32_t chunk_bytes = (uint32_t)(128 * mp8);

  if (warp == 4) {
    // ---------------- producer: chunks of every block in use order, each asked of L2
    // kX3Prefetch chunks before its copy
    if (lane == 0) {
      auto chunk_src = [&](int64_t it) {
        const int st = (int)(it / nck), c = (int)(it - (int64_t)st * nck);
        const int j = st < rows ? st : 2 * rows - 2 - st;
        return Fs + j * slot_floats + (int64_t)c * 32 * mp8;
      };
      for (int64_t it = 0; it < min(total, (int64_t)kX3Prefetch); ++it) prefetch_l2(chunk_src(it), chunk_bytes);
      int64_t issued = 0;
      bool ok = true;
      for (int64_t it = 0; it < total && ok; ++it) {
        if (it + kX3Prefetch < total) prefetch_l2(chunk_src(it + kX3Prefetch), chunk_bytes);
        const int slot = (int)(it % NS);
        const uint32_t ph = (uint32_t)((it / NS) & 1);
        if (!tc::bar_spin(&empty[slot], ph ^ 1u, abort_flag)) { ok = false; break; }
        bar_expect(&full[slot], chunk_bytes);
        bulk_copy(ring + (size_t)slot * stage_bytes, chunk_src(it), chunk_bytes, &full[slot]);
        issued = it + 1;
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(status, ST_TIMEOUT);
      }
      // no copy may still be landing when the CTA exits
      for (int64_t it = max((int64_t)0, issued - NS); it < issued; ++it)
        tc::bar_wait(&full[it % NS], (uint32_t)((it / NS) & 1), abort_flag);
    }
    return;
  }

  if (warp == 5) {
    // ---------------- MMA issuer (one thread); the warp owns the tensor memory
    if (lane == 0) {
      // D f32, A and B tf32, both K-major, N = m rounded up to 16, M = 128
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(mp16 >> 3) << 17) | ((128u >> 4) << 24);
      const uint32_t a1 = tc::su32(A1), a2 = tc::su32(A2), pl = (uint32_t)(32 * mp8);
      int64_t it = 0;
      bool ok = true;
      for (int st = 0; st < nsteps && ok; ++st) {
        const uint32_t d = tmem + (uint32_t)(st & 1) * X3_HALF;
        for (int c = 0; c < nck; ++c, ++it) {
          if ((c & 3) == 0) {   // the next 32 columns of V (this step's K range) are written
            if (!tc::bar_spin(&aready[c >> 2], (uint32_t)(st & 1), abort_flag)) { ok = false; break; }
            tc::fence_after();
          }
          const int slot = (int)(it % NS);
          if (!tc::bar_spin(&full[slot], (uint32_t)((it / NS) & 1), abort_flag)) { ok = false; break; }
          const uint32_t sb = tc::su32(ring + (size_t)slot * stage_bytes);
          const uint64_t da1 = tc::mdesc(a1 + (uint32_t)c * 2 * kX3Lbo, kX3Lbo, asbo);
          const uint64_t da2 = tc::mdesc(a2 + (uint32_t)c * 2 * kX3Lbo, kX3Lbo, asbo);
          mma_tf32(d, da1, tc::mdesc(sb, 128, 256), idesc, c > 0 ? 1u : 0u);
          mma_tf32(d, da2, tc::mdesc(sb + pl, 128, 256), idesc, 1u);
          mma_tf32(d, da1, tc::mdesc(sb + 2 * pl, 128, 256), idesc, 1u);
          mma_tf32(d, da2, tc::mdesc(sb + 3 * pl, 128, 256), idesc, 1u);
          tc::mma_commit(&empty[slot]);   // the stage is free once these MMAs have read it
        }
        if (!ok) break;
        tc::mma_commit(dfull);
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(status, ST_TIMEOUT);
      }
      tc::mma_commit(fin);                          // arrives once every MMA issued above is done
      tc::bar_wait(fin, 0, abort_flag);
      tc::bar_wait(edone, 0, abort_flag);           // the epilogue has finished reading tensor memory
    }
    __syncwarp();
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)X3_TMEM_COLS)
                 : "memory");
    return;
  }

  // ---------------- epilogue: lane (part, s) of warp w; right-hand side src = 8w + s.
  // After the two lane exchanges this thread holds Yr and Yi of src for the 8 columns
  // coff .. coff+7 of each 32-column group (parts 0, 2, 1, 3 -> columns 0, 8, 16, 24).
  const int part = lane >> 3, sl = lane & 7, src = 8 * warp + sl;
  const int coff = 16 * (part & 1) + 8 * (part >> 1);
  const bool odd = (part & 1) != 0, up = part >= 2;
  const bool live = r0 + src < nrhs;
  const double2 *rgs = rg + (int64_t)(live ? r0 + src : 0) * vec_stride;
  float2 *stg = staging + (int64_t)(live ? r0 + src : 0) * stg_stride + s.soff;
  auto owned_x = [&](int a) { return a < m && s.ex0 + a >= s.ox0 && s.ex0 + a < s.ox1; };
  // residual of grid row gy at columns k0 .. k0+7 (zero outside the owned box, past m, or for idle sources)
  auto load_rho = [&](int gy, int k0, float2 *v) {
    const bool owny = live && gy >= s.oy0 && gy < s.oy1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int a = k0 + i;
      v[i] = make_float2(0.f, 0.f);
      if (owny && owned_x(a)) {
        const double2 x = rgs[(int64_t)gy * NX + s.ex0 + a];
        v[i] = make_float2((float)x.x, (float)x.y);
      }
    }
  };
  // V_0 = rho_0 (zero in the K padding columns m <= a < mp8)
  for (int g = 0; g < ngrp; ++g) {
    const int k0 = 32 * g + coff;
    if (k0 < mp8) {
      float2 v[8];
      load_rho(s.ey0, k0, v);
      put_v8(A1, A2, asbo, warp, sl, k0, v);
    }
    tc::fence_async_smem();
    tc::fence_before();
    bar_arrive(&aready[g]);
  }

  for (int st = 0; st < nsteps; ++st) {
    const bool fwd = st < rows;
    const int j = fwd ? st : 2 * rows - 2 - st;
    // the next step's coupling: forward rho_{j+1} - L_{j+1} w_j, backward U_{jn} x_{jn+1}
    const int sn = st + 1;
    const bool has_next = sn < nsteps;
    const bool nfwd = sn < rows;
    const int jn = nfwd ? sn : 2 * rows - 2 - sn;
    float2 cpl = make_float2(0.f, 0.f);
    if (has_next) {
      const double2 c = nfwd ? pool[s.aoff + 2 * m + 1 + rows + jn] : pool[s.aoff + 2 * m + 1 + rows + jn + 1];
      cpl = make_float2((float)c.x, (float)c.y);
    }
    float2 pre[X3_GROUPS][8];
#pragma unroll
    for (int g = 0; g < X3_GROUPS; ++g) {
      const int k0 = 32 * g + coff;
#pragma unroll
      for (int i = 0; i < 8; ++i) pre[g][i] = make_float2(0.f, 0.f);
      if (g < ngrp && k0 < mp8) {
        if (!fwd) {
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (live && k0 + i < m) pre[g][i] = stg[(int64_t)j * m + k0 + i];
        } else if (has_next && nfwd) {
          load_rho(s.ey0 + jn, k0, pre[g]);
        }
      }
    }
    const bool got = __all_sync(0xffffffffu, tc::bar_spin(dfull, (uint32_t)(st & 1), abort_flag));
    if (!got) {
      if (lane == 0) {
        *abort_flag = 1;
        atomicOr(status, ST_TIMEOUT);
      }
      break;
    }
    tc::fence_after();
    const uint32_t dcol = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(st & 1) * X3_HALF;
#pragma unroll
    for (int g = 0; g < X3_GROUPS; ++g) {
      if (g >= ngrp) break;
      const int k0 = 32 * g + coff;
      const bool colok = k0 < mp8;
      float v[32];
      tmem_ld32(dcol + (uint32_t)(32 * g), v);   // warp-collective
      // hi + lo parts (lanes l, l ^ 8): keep 16 of the 32 columns
      float h[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const float x = odd ? v[c] : v[16 + c];
        const float y = __shfl_xor_sync(0xffffffffu, x, 8);
        h[c] = (odd ? v[16 + c] : v[c]) + y;
      }
      // real and imaginary parts (lanes l, l ^ 16): keep 8 columns, both parts
      float2 y8[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float x = up ? h[c] : h[8 + c];
        const float y = __shfl_xor_sync(0xffffffffu, x, 16);
        const float own = up ? h[8 + c] : h[c];
        y8[c] = up ? make_float2(y, own) : make_float2(own, y);
      }
      if (colok) {
        float2 nv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int a = k0 + i;
          const float2 out = fwd ? y8[i] : csub(pre[g][i], y8[i]);
          if (live && a < m) stg[(int64_t)j * m + a] = out;
          const float2 lc = cmul(lA[a], cpl);   // L_{jn} or U_{jn} entry of row a (zero past m)
          nv[i] = nfwd ? cfms(lc, out, pre[g][i]) : cmul(lc, out);
          if (a >= m) nv[i] = make_float2(0.f, 0.f);
        }
        if (has_next) put_v8(A1, A2, asbo, warp, sl, k0, nv);
      }
      if (has_next) {
        tc::fence_async_smem();
        tc::fence_before();
        bar_arrive(&aready[g]);
      }
    }
  }
  tc::fence_before();
  bar_arrive(edone);
}

// One CTA per SM (the two accumulators take all 512 tensor-memory columns); ring stages
// as many as fit beside the A operands, at least two.
cudaError_t launch_subst_x3(hd_ctx *ctx, const double2 *r, int nrhs, int64_t vec_stride, void *staging,
                            int64_t stg_stride, cudaStream_t st) {
  const int mp8max = (ctx->max_m + 7) & ~7;
  if (mp8max > kMaxBoxWidthX3) return cudaErrorInvalidValue;
  const int groups = (nrhs + X3_NR - 1) / X3_NR;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int ns = 2;
  while (ns < 8 && subst_x3_smem(ns + 1, mp8max) <= (size_t)optin) ++ns;
  size_t smem = subst_x3_smem(ns, mp8max);
  if (smem > (size_t)optin) return cudaErrorInvalidValue;
  smem = std::max(smem, (size_t)optin / 2 + 1024);   // keeps a second CTA off the SM
  cudaError_t e = allow_smem(k_subst_x3, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(groups, ctx->nsub);
  k_subst_x3<<<grid, X3_THREADS, smem, st>>>(ctx->d_subs, ctx->d_lpool, reinterpret_cast<const float *>(ctx->factor),
                                             r, ctx->NX, vec_stride, reinterpret_cast<float2 *>(staging), stg_stride,
                                             nrhs, ns, mp8max, ctx->d_status);
  return cudaGetLastError();
}

}  // namespace hd
