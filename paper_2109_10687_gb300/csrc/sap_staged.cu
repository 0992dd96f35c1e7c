// SAP half-sweep kernel for 4^4 domains with the domain's links and C_inv
// held in shared memory in float32 (Sec. 3 of arXiv:2109.10687, Algorithms 1
// and 2; the arithmetic is that of sap.cu's generic kernel).
//
// One CTA of 512 threads per domain, two threads per site.  Thread half 0 of
// a site takes the hops in x and y and the upper chiral block (spins 0, 1),
// half 1 the hops in z and t and the lower block (spins 2, 3).  After its
// hops each thread hands the partial sum of the other chirality to its
// partner through shared memory, then applies its own 6x6 block of C_inv and
// updates its half of the iterate.  The domain shape is fixed at compile time
// (strides 1, 4, 16, 64).
//
// Staging (per domain, identical element order in global and shared memory):
//   links : [mu 4][site 256][9]        complex (float2 / __half2)
//   C_inv : [block 2][site 256][18]    complex pairs of the packed block
// float32 storage: one thread arms an mbarrier and two cp.async.bulk copies
// bring both blocks in while the threads evaluate the surface hops; float16
// storage: every thread converts a share of the block to float32 on the way
// into shared memory, once per launch instead of once per use.
//
// Shared memory: x iterate 24 KB + links 72 KB + C_inv 72 KB + exchange 24 KB.

#include <type_traits>

#include "qcd_internal.cuh"

namespace qcd {

constexpr int SP_THREADS = 512;
constexpr int LINK32_BYTES = 4 * 256 * 9 * 8;   // 73728 per domain
constexpr int CLOV32_BYTES = 2 * 256 * 36 * 4;  // 73728 per domain
constexpr int LINK16_BYTES = 4 * 256 * 9 * 4;   // 36864
constexpr int CLOV16_BYTES = 2 * 256 * 36 * 2;  // 36864
constexpr int SX_BYTES = 6 * 256 * 16;          // 24576
constexpr int SMEM_BYTES = SX_BYTES + LINK32_BYTES + CLOV32_BYTES + SX_BYTES + 16;

template <bool HALF>
using StageSpinor = typename std::conditional<HALF, F16Spinor, F32Spinor>::type;

template <bool HALF>
struct StagedArgs {
  Geom g;
  int colour, n_jac, do_surface, do_update, nrhs;
  float kappa;
  StageSpinor<HALF> s_in, s_out, x;
  F32Spinor b;
  const void* links;  // staging layout, all domains (float2 or __half2)
  const void* clov;   // staging layout, all domains
  int* status;        // set to QCD_ERR_TIMEOUT if a wait gives up
};

// ---------------------------------------------------------------------------
// mbarrier + bulk copy (PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: at most 2^22 polls (each try_wait itself suspends for a
// while); returns false when it gives up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (int i = 0; i < (1 << 22); ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// ---------------------------------------------------------------------------
// shared-memory accessors
// ---------------------------------------------------------------------------
template <int MU>
__device__ __forceinline__ int lc(int s) { return (s >> (2 * MU)) & 3; }

// x iterate: float4 group k holds complex components 2k, 2k + 1
// (component = spin * 3 + colour)
__device__ __forceinline__ void sx_load(const float4* sx, int site, Spinor<float>& p) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 v = sx[k * 256 + site];
    p.v[(2 * k) / 3][(2 * k) % 3] = make_cx(v.x, v.y);
    p.v[(2 * k + 1) / 3][(2 * k + 1) % 3] = make_cx(v.z, v.w);
  }
}
// chirality h (0: spins 0, 1 = groups 0..2; 1: spins 2, 3 = groups 3..5)
__device__ __forceinline__ void sx_store_half(float4* sx, int site, int h, const cx<float> a[6]) {
#pragma unroll
  for (int k = 0; k < 3; ++k)
    sx[(3 * h + k) * 256 + site] = make_float4(a[2 * k].re, a[2 * k].im, a[2 * k + 1].re, a[2 * k + 1].im);
}
__device__ __forceinline__ void sx_load_half(const float4* sx, int site, int h, cx<float> a[6]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 v = sx[(3 * h + k) * 256 + site];
    a[2 * k] = make_cx(v.x, v.y);
    a[2 * k + 1] = make_cx(v.z, v.w);
  }
}

__device__ __forceinline__ SU3<float> slink(const float2* sl, int mu, int site) {
  const float2* p = sl + (mu * 256 + site) * 9;
  SU3<float> u;
#pragma unroll
  for (int e = 0; e < 9; ++e) u.m[e / 3][e % 3] = make_cx(p[e].x, p[e].y);
  return u;
}

// apply the packed Hermitian block `blk` of C_inv at `site` to a[6]
__device__ __forceinline__ void sclover(const float* sc, int blk, int site, cx<float> a[6]) {
  const float4* p = reinterpret_cast<const float4*>(sc + (blk * 256 + site) * 36);
  CloverBlockF32 cb;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float4 v = p[k];
    cb.r[4 * k] = v.x; cb.r[4 * k + 1] = v.y; cb.r[4 * k + 2] = v.z; cb.r[4 * k + 3] = v.w;
  }
  cx<float> y[6];
  herm6_mul<float>(cb, a, y);
#pragma unroll
  for (int i = 0; i < 6; ++i) a[i] = y[i];
}

// acc += both intra-domain hops of direction MU
template <int MU>
__device__ __forceinline__ void sp_intra(const float4* sx, const float2* sl, int s, Spinor<float>& acc) {
  constexpr int step = 1 << (2 * MU);
  const int c = lc<MU>(s);
  if (c < 3) {
    Spinor<float> p;
    sx_load(sx, s + step, p);
    HalfSpinor<float> h, uh;
    project<MU, -1>(p, h);
    su3_mul(slink(sl, MU, s), h, uh);
    accumulate<MU, -1>(acc, uh);
  }
  if (c > 0) {
    Spinor<float> p;
    sx_load(sx, s - step, p);
    HalfSpinor<float> h, uh;
    project<MU, +1>(p, h);
    su3_dag_mul(slink(sl, MU, s - step), h, uh);
    accumulate<MU, +1>(acc, uh);
  }
}

// link of the staging layout in global memory (any domain)
template <bool HALF>
__device__ __forceinline__ SU3<float> glink(const void* links, int dom, int mu, int site) {
  SU3<float> u;
  if (HALF) {
    const __half2* p = reinterpret_cast<const __half2*>(links) + ((size_t)(dom * 4 + mu) * 256 + site) * 9;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const float2 v = __half22float2(p[e]);
      u.m[e / 3][e % 3] = make_cx(v.x, v.y);
    }
  } else {
    const float2* p = reinterpret_cast<const float2*>(links) + ((size_t)(dom * 4 + mu) * 256 + site) * 9;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const float2 v = __ldg(p + e);
      u.m[e / 3][e % 3] = make_cx(v.x, v.y);
    }
  }
  return u;
}

// acc += both domain-leaving hops of direction MU (x and links from memory)
template <int MU, bool HALF, typename SIO>
__device__ __forceinline__ void sp_inter(const Geom& g, const SIO& x, const void* links, int dom, int s, int rhs_off,
                                         Spinor<float>& acc) {
  constexpr int step = 1 << (2 * MU);
  const int c = lc<MU>(s);
  if (c == 3) {
    const int nd = __ldg(g.nbr + dom * 8 + 2 * MU);
    const int sign = ((__ldg(g.tflag + dom) >> (2 * MU)) & 1) ? g.bc_t : 1;
    Spinor<float> p;
    x.load(g, nd + rhs_off, s - 3 * step, p);
    HalfSpinor<float> h, uh;
    project<MU, -1>(p, h);
    su3_mul(glink<HALF>(links, dom, MU, s), h, uh);
    if (sign < 0) scale_half(uh, -1.0f);
    accumulate<MU, -1>(acc, uh);
  }
  if (c == 0) {
    const int nd = __ldg(g.nbr + dom * 8 + 2 * MU + 1);
    const int sign = ((__ldg(g.tflag + dom) >> (2 * MU + 1)) & 1) ? g.bc_t : 1;
    const int ns = s + 3 * step;
    Spinor<float> p;
    x.load(g, nd + rhs_off, ns, p);
    HalfSpinor<float> h, uh;
    project<MU, +1>(p, h);
    su3_dag_mul(glink<HALF>(links, nd, MU, ns), h, uh);
    if (sign < 0) scale_half(uh, -1.0f);
    accumulate<MU, +1>(acc, uh);
  }
}

// chirality h of a spinor (h is warp-uniform; both branches use constant
// register indices so the spinor stays in registers)
__device__ __forceinline__ void take_half(const Spinor<float>& a, int h, cx<float> out[6]) {
  if (h == 0) {
#pragma unroll
    for (int i = 0; i < 6; ++i) out[i] = a.v[i / 3][i % 3];
  } else {
#pragma unroll
    for (int i = 0; i < 6; ++i) out[i] = a.v[2 + i / 3][i % 3];
  }
}

// Hand the other chirality of `acc` to the partner thread and take its share
// of ours; returns this thread's chirality summed over all eight directions.
// Contains one __syncthreads, after which no thread reads the x iterate of the
// current sweep any more.
__device__ __forceinline__ void exchange(float4* sxch, int s, int h, const Spinor<float>& acc, cx<float> mine[6]) {
  cx<float> give[6];
  take_half(acc, 1 - h, give);
  take_half(acc, h, mine);
  sx_store_half(sxch, s, 1 - h, give);
  __syncthreads();
  cx<float> got[6];
  sx_load_half(sxch, s, h, got);
#pragma unroll
  for (int i = 0; i < 6; ++i) mine[i] = mine[i] + got[i];
}

template <bool HALF>
__global__ void __launch_bounds__(SP_THREADS, 1) sap_split_kernel(StagedArgs<HALF> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  float4* sx = reinterpret_cast<float4*>(smem);
  float2* sl = reinterpret_cast<float2*>(smem + SX_BYTES);
  float* sc = reinterpret_cast<float*>(smem + SX_BYTES + LINK32_BYTES);
  float4* sxch = reinterpret_cast<float4*>(smem + SX_BYTES + LINK32_BYTES + CLOV32_BYTES);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SX_BYTES + LINK32_BYTES + CLOV32_BYTES + SX_BYTES);
  const Geom& g = a.g;
  const int tid = threadIdx.x;
  const int h = tid >> 8;  // 0: x, y hops + upper block; 1: z, t hops + lower block
  const int s = tid & 255;
  const int dom = a.colour * g.nhalf + blockIdx.x;

  if (HALF) {
    // float16 staging -> float32 shared memory, converted on the way in
    const uint4* gl = reinterpret_cast<const uint4*>(a.links) + (size_t)dom * (LINK16_BYTES / 16);
    const uint4* gc = reinterpret_cast<const uint4*>(a.clov) + (size_t)dom * (CLOV16_BYTES / 16);
    float4* dl = reinterpret_cast<float4*>(sl);
    float4* dc = reinterpret_cast<float4*>(sc);
    for (int k = tid; k < LINK16_BYTES / 16; k += SP_THREADS) {
      const uint4 v = __ldg(gl + k);
      const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
      const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
      const float2 f2 = __half22float2(*reinterpret_cast<const __half2*>(&v.z));
      const float2 f3 = __half22float2(*reinterpret_cast<const __half2*>(&v.w));
      dl[2 * k] = make_float4(f0.x, f0.y, f1.x, f1.y);
      dl[2 * k + 1] = make_float4(f2.x, f2.y, f3.x, f3.y);
    }
    for (int k = tid; k < CLOV16_BYTES / 16; k += SP_THREADS) {
      const uint4 v = __ldg(gc + k);
      const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
      const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
      const float2 f2 = __half22float2(*reinterpret_cast<const __half2*>(&v.z));
      const float2 f3 = __half22float2(*reinterpret_cast<const __half2*>(&v.w));
      dc[2 * k] = make_float4(f0.x, f0.y, f1.x, f1.y);
      dc[2 * k + 1] = make_float4(f2.x, f2.y, f3.x, f3.y);
    }
  } else if (tid == 0) {
    mbar_init(bar, 1);
    mbar_expect_tx(bar, LINK32_BYTES + CLOV32_BYTES);
    bulk_copy_g2s(sl, (const unsigned char*)a.links + (size_t)dom * LINK32_BYTES, LINK32_BYTES, bar);
    bulk_copy_g2s(sc, (const unsigned char*)a.clov + (size_t)dom * CLOV32_BYTES, CLOV32_BYTES, bar);
  }

  for (int r = 0; r < a.nrhs; ++r) {
    const int rhs_off = r * g.ndom;
    const int domr = dom + rhs_off;
    cx<float> src[6];  // this thread's chirality of s_c (after the surface term)
    {
      Spinor<float> sfull;
      a.s_in.load(g, domr, s, sfull);
      take_half(sfull, h, src);
    }
    Spinor<float> acc;
    zero(acc);
    if (a.do_surface) {
      if (h == 0) {
        sp_inter<0, HALF>(g, a.x, a.links, dom, s, rhs_off, acc);
        sp_inter<1, HALF>(g, a.x, a.links, dom, s, rhs_off, acc);
      } else {
        sp_inter<2, HALF>(g, a.x, a.links, dom, s, rhs_off, acc);
        sp_inter<3, HALF>(g, a.x, a.links, dom, s, rhs_off, acc);
      }
    }
    if (r == 0) {
      __syncthreads();  // staging (float16) / barrier initialisation (float32) visible
      if (!HALF) {
        const bool ok = mbar_wait_bounded(bar, 0);
        if (__syncthreads_or(!ok)) {
          // a wait gave up: record it, give the copies one more bounded wait
          // and leave (the decision is uniform across the CTA)
          if (tid == 0) atomicExch(a.status, QCD_ERR_TIMEOUT);
          if (!ok) mbar_wait_bounded(bar, 0);
          return;
        }
      }
    }
    if (a.do_surface) {
      cx<float> mine[6];
      exchange(sxch, s, h, acc, mine);
      sclover(sc, h, s, mine);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        src[i].re = fmaf(a.kappa, mine[i].re, src[i].re);
        src[i].im = fmaf(a.kappa, mine[i].im, src[i].im);
      }
    }
    sx_store_half(sx, s, h, src);
    __syncthreads();

    cx<float> xk[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) xk[i] = src[i];
    const int napp = a.n_jac + (a.do_update ? 1 : 0);
    for (int it = 0; it < napp; ++it) {
      zero(acc);
      if (h == 0) {
        sp_intra<0>(sx, sl, s, acc);
        sp_intra<1>(sx, sl, s, acc);
      } else {
        sp_intra<2>(sx, sl, s, acc);
        sp_intra<3>(sx, sl, s, acc);
      }
      cx<float> mine[6];
      exchange(sxch, s, h, acc, mine);  // all reads of sx for this sweep are done
      sclover(sc, h, s, mine);
      if (it < a.n_jac) {
        // x_k = s_c + kappa C_inv H_cc x_{k-1}
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          xk[i].re = fmaf(a.kappa, mine[i].re, src[i].re);
          xk[i].im = fmaf(a.kappa, mine[i].im, src[i].im);
        }
        sx_store_half(sx, s, h, xk);
        __syncthreads();
      } else {
        // s_c + b_c - x_c + kappa C_inv H_cc x_c, assembled in the exchange buffer
        Spinor<float> bfull;
        a.b.load(g, domr, s, bfull);
        cx<float> bh[6], so[6];
        take_half(bfull, h, bh);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          so[i].re = fmaf(a.kappa, mine[i].re, src[i].re + bh[i].re - xk[i].re);
          so[i].im = fmaf(a.kappa, mine[i].im, src[i].im + bh[i].im - xk[i].im);
        }
        __syncthreads();  // partners have read their exchange halves
        sx_store_half(sxch, s, h, so);
        __syncthreads();
      }
    }
    // stores: half 0 writes x (complete in sx), half 1 writes s (complete in sxch)
    if (h == 0) {
      Spinor<float> xf;
      sx_load(sx, s, xf);
      a.x.store(g, domr, s, xf);
    } else if (a.do_update) {
      Spinor<float> sf;
      sx_load(sxch, s, sf);
      a.s_out.store(g, domr, s, sf);
    }
    __syncthreads();  // shared buffers free for the next right-hand side
  }
}

// ---------------------------------------------------------------------------
// staging layouts, built from the internal float64 layouts
// ---------------------------------------------------------------------------
__global__ void build_link_stage_kernel(Geom g, const double2* u64, __half2* l16, float2* l32) {
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gid >= g.vol * 4) return;
  const int s = (int)(gid & 255);
  const int mu = (int)((gid >> 8) & 3);
  const int dom = (int)(gid >> 10);
  for (int e = 0; e < 9; ++e) {
    const double2 v = u64[(((size_t)((dom * 4 + mu) * 9 + e)) << 8) + s];
    const size_t o = ((size_t)(dom * 4 + mu) * 256 + s) * 9 + e;
    l16[o] = __floats2half2_rn((float)v.x, (float)v.y);
    l32[o] = make_float2((float)v.x, (float)v.y);
  }
}

__global__ void build_clover_stage_kernel(Geom g, const double2* c64, __half2* c16, float2* c32) {
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gid >= g.vol) return;
  const int s = (int)(gid & 255);
  const int dom = (int)(gid >> 8);
  for (int b = 0; b < 2; ++b)
    for (int k = 0; k < 18; ++k) {
      const double2 v = c64[(((size_t)(dom * 36 + 18 * b + k)) << 8) + s];
      const size_t o = ((size_t)(dom * 2 + b) * 256 + s) * 18 + k;
      c16[o] = __floats2half2_rn((float)v.x, (float)v.y);
      c32[o] = make_float2((float)v.x, (float)v.y);
    }
}

bool sap_staged_available(const qcd_ctx* ctx) {
  const Geom& g = ctx->geom;
  return g.d[0] == 4 && g.d[1] == 4 && g.d[2] == 4 && g.d[3] == 4 && ctx->st_link16 && ctx->st_clov16;
}

void build_sap_staging(qcd_ctx* ctx, cudaStream_t st) {
  const Geom& g = ctx->geom;
  if (!(g.d[0] == 4 && g.d[1] == 4 && g.d[2] == 4 && g.d[3] == 4)) return;
  const size_t nd = (size_t)g.ndom;
  if (!ctx->st_link16) {
    QCD_CUDA_CHECK(cudaMalloc(&ctx->st_link16, nd * LINK16_BYTES));
    QCD_CUDA_CHECK(cudaMalloc(&ctx->st_link32, nd * LINK32_BYTES));
    QCD_CUDA_CHECK(cudaMalloc(&ctx->st_clov16, nd * CLOV16_BYTES));
    QCD_CUDA_CHECK(cudaMalloc(&ctx->st_clov32, nd * CLOV32_BYTES));
    QCD_CUDA_CHECK(cudaFuncSetAttribute(sap_split_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        SMEM_BYTES));
    QCD_CUDA_CHECK(cudaFuncSetAttribute(sap_split_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        SMEM_BYTES));
  }
  LaunchScope ls(ctx, QCD_KC_OTHER, st);
  build_link_stage_kernel<<<grid_for(g.vol * 4, 256), 256, 0, st>>>(g, ctx->u64, (__half2*)ctx->st_link16,
                                                                    (float2*)ctx->st_link32);
  build_clover_stage_kernel<<<grid_for(g.vol, 256), 256, 0, st>>>(g, ctx->cinv64, (__half2*)ctx->st_clov16,
                                                                  (float2*)ctx->st_clov32);
  check_launch();
}

template <bool HALF>
static void staged_sequence(qcd_ctx* ctx, StageSpinor<HALF> s_first_in, StageSpinor<HALF> s, StageSpinor<HALF> x,
                            F32Spinor b, int nrhs, int n_sap, int n_jac, cudaStream_t st) {
  StagedArgs<HALF> a;
  a.g = ctx->geom;
  a.nrhs = nrhs;
  a.n_jac = n_jac;
  a.kappa = (float)ctx->kappa;
  a.b = b;
  a.x = x;
  a.s_out = s;
  a.links = HALF ? ctx->st_link16 : ctx->st_link32;
  a.clov = HALF ? ctx->st_clov16 : ctx->st_clov32;
  a.status = ctx->d_status;
  for (int sweep = 0; sweep <= n_sap; ++sweep) {
    a.s_in = sweep == 0 ? s_first_in : s;
    a.do_update = sweep == n_sap ? 0 : 1;
    for (int colour = 0; colour < 2; ++colour) {
      a.colour = colour;
      a.do_surface = (sweep == 0 && colour == 0) ? 0 : 1;
      LaunchScope ls(ctx, QCD_KC_SAP_BLOCK, st);
      sap_split_kernel<HALF><<<ctx->geom.nhalf, SP_THREADS, SMEM_BYTES, st>>>(a);
      check_launch();
    }
  }
}

void sap_staged_sequence_f32(qcd_ctx* ctx, F32Spinor s_first_in, F32Spinor s, F32Spinor x, F32Spinor b, int nrhs,
                             int n_sap, int n_jac, cudaStream_t st) {
  staged_sequence<false>(ctx, s_first_in, s, x, b, nrhs, n_sap, n_jac, st);
}
void sap_staged_sequence_f16(qcd_ctx* ctx, F16Spinor s_first_in, F16Spinor s, F16Spinor x, F32Spinor b, int nrhs,
                             int n_sap, int n_jac, cudaStream_t st) {
  staged_sequence<true>(ctx, s_first_in, s, x, b, nrhs, n_sap, n_jac, st);
}

}  // namespace qcd
