// SAP half-sweep kernel for 4^4 domains with the domain's links and C_inv
// staged in shared memory by bulk asynchronous copies (Sec. 3 of
// arXiv:2109.10687, Algorithms 1 and 2; the arithmetic is that of
// sap.cu's generic kernel).
//
// One CTA per domain, one thread per site, the domain shape fixed at compile
// time (strides 1, 4, 16, 64).  At entry one thread arms an mbarrier and
// issues two cp.async.bulk copies: the domain's links and its C_inv, each a
// contiguous block of a staging layout built for this kernel.  The launches
// of one M_SAP use programmatic dependent launch: these copies are issued
// before the kernel waits for the previous launch.  After that wait the
// same thread issues a third copy, the domain's halo block (below), and the
// threads read their s; they then wait (bounded) on the copies and run the
// surface term, every Jacobi sweep and the residual update from shared
// memory.
//
// Halo.  The surface term of a colour-c launch needs, for each hop that
// enters the domain, U P x of the neighbouring (other-colour) domain's
// iterate.  The launch that computed that iterate still holds it, and its
// own links, in shared memory, so it finishes the work there: for each of
// its face sites it writes the half spinor the neighbour needs into the
// neighbour's halo slots, U^dag P+ x for a backward hop (complete) and P- x
// for a forward hop (the receiver multiplies by its own link U, which it has
// staged).  The receiving launch brings its halo block in with one bulk copy
// and needs no neighbour lookups.  This is the exchange of Sec. 4.1, done
// through memory.
//
//   staging layouts per domain (global = shared):
//     links  f16: __half2 [mu 4][site 256][10]    40 B per link (9 + pad), 8-byte reads
//            f32: float2  [mu 4][site 256][9]     72 B per link, 8-byte reads
//     C_inv  f16: uint4   [site 256][9]           two blocks of 36 halves
//            f32: float4  [site 256][19]          two blocks of 36 floats + pad
//   (these site strides make each warp's reads free of shared-memory bank
//   conflicts)
//
// sap_flow_kernel runs the same half-sweeps, a whole M_SAP, in one launch of
// resident CTAs ordered by per-domain flags (an autotuner shape).
//
// Shared memory: f16 103 KB (two CTAs per SM), f32 176 KB (one CTA per SM).
// Three mbarriers: the staged links and the staged C_inv (once per item a
// CTA runs; the surface term needs only the links, so it starts before
// C_inv has landed) and the halo copy (once per right-hand side of an item
// with a surface term; its phase counts those copies).

#include <cstdio>
#include <cstring>
#include <type_traits>
#include <vector>

#include "qcd_internal.cuh"

namespace qcd {

constexpr int ST_THREADS = 256;
constexpr int C16_U4 = 9;    // uint4 per site, f16 C_inv
constexpr int L16_H2 = 10;   // half2 per link, f16 links (9 + 1 pad)
constexpr int C32_F4 = 19;   // float4 per site, f32 C_inv

template <bool HALF>
struct StageT;

template <>
struct StageT<true> {
  static constexpr int LINK_BYTES = 4 * 256 * L16_H2 * 4;  // 40960
  static constexpr int CLOV_BYTES = 256 * C16_U4 * 16;     // 36864
  using SIO = F16Spinor;
  // a link is 9 half2 padded to 10 (40 bytes): five 8-byte reads, and the
  // 10-word site stride keeps a half warp's 8-byte reads on distinct banks
  __device__ static SU3<float> link(const unsigned char* base, int mu, int site) {
    const uint2* p = reinterpret_cast<const uint2*>(base) + (mu * 256 + site) * (L16_H2 / 2);
    SU3<float> u;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const uint2 w = p[k];
      const float2 v0 = __half22float2(*reinterpret_cast<const __half2*>(&w.x));
      u.m[(2 * k) / 3][(2 * k) % 3] = make_cx(v0.x, v0.y);
      if (2 * k + 1 < 9) {
        const float2 v1 = __half22float2(*reinterpret_cast<const __half2*>(&w.y));
        u.m[(2 * k + 1) / 3][(2 * k + 1) % 3] = make_cx(v1.x, v1.y);
      }
    }
    return u;
  }
  // the two blocks are 36 halves each, back to back in 9 uint4 (144 bytes,
  // an odd number of 16-byte units per site: a quarter warp's 16-byte reads
  // fall on distinct bank groups); block 0 is uint4 0-3 and the first 8
  // bytes of uint4 4, block 1 the last 8 bytes of uint4 4 and uint4 5-8
  __device__ static void clover_block(const unsigned char* base, int site, int b, CloverBlockF32& blk) {
    const uint4* p = reinterpret_cast<const uint4*>(base) + site * C16_U4;
    unsigned w[18];
    const uint2 mid = reinterpret_cast<const uint2*>(p + 4)[b];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint4 v = p[b == 0 ? k : 5 + k];
      const int o = b == 0 ? 4 * k : 2 + 4 * k;
      w[o] = v.x; w[o + 1] = v.y; w[o + 2] = v.z; w[o + 3] = v.w;
    }
    w[b == 0 ? 16 : 0] = mid.x;
    w[b == 0 ? 17 : 1] = mid.y;
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      const float2 v = __half22float2(*reinterpret_cast<const __half2*>(&w[k]));
      blk.r[2 * k] = v.x;
      blk.r[2 * k + 1] = v.y;
    }
  }
};

template <>
struct StageT<false> {
  static constexpr int LINK_BYTES = 4 * 256 * 9 * 8;       // 73728
  static constexpr int CLOV_BYTES = 256 * C32_F4 * 16;     // 77824
  using SIO = F32Spinor;
  __device__ static SU3<float> link(const unsigned char* base, int mu, int site) {
    const float2* p = reinterpret_cast<const float2*>(base) + (mu * 256 + site) * 9;
    SU3<float> u;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const float2 v = p[e];
      u.m[e / 3][e % 3] = make_cx(v.x, v.y);
    }
    return u;
  }
  __device__ static void clover_block(const unsigned char* base, int site, int b, CloverBlockF32& blk) {
    const float4* p = reinterpret_cast<const float4*>(base) + site * C32_F4 + 9 * b;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float4 v = p[k];
      blk.r[4 * k] = v.x; blk.r[4 * k + 1] = v.y; blk.r[4 * k + 2] = v.z; blk.r[4 * k + 3] = v.w;
    }
  }
};

template <bool HALF, typename SIO>
struct StagedArgs {
  Geom g;
  int colour, n_jac, do_surface, do_update, nrhs;
  float kappa;
  SIO s_in, s_out, x;   // vectors: float16 or float32 storage, independent of HALF
  F32Spinor b;
  F32Spinor s_in32;      // if set: the sweep's input is read from this float32 field instead of s_in
  F32Spinor x_out32;     // if set: the iterate is also stored to this float32 field
  int x_store;           // store the iterate in x (the result of M_SAP)
  int do_halo;           // write the neighbours' halo (0 in the last launch)
  float4* halo;          // [rhs][domain][face 8][3][64] float4, face = 2 MU + side
  const unsigned char* links;  // staging layout, all domains
  const unsigned char* clov;
  int* status;                 // word 0: set to QCD_ERR_TIMEOUT if a wait gives up
  int extra_tx;                // testing: bytes the staging wait expects beyond its copies
  int extra_htx;               // testing: bytes the halo wait expects beyond its copy
  const int* skip;             // if set and nonzero: this lattice has stopped iterating (ragged batch)
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
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: gives up (returns false) after half a second of polling, or
// 2^24 polls, whichever comes first.  The copies it waits for take
// microseconds.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < (1 << 24); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255) == 255 && global_ns() - t0 > 500000000ull) return false;
  }
  return false;
}

// ---------------------------------------------------------------------------
// hops
// ---------------------------------------------------------------------------
// local coordinates of a 4^4 site: x = s & 3, y = (s >> 2) & 3, z = (s >> 4) & 3, t = s >> 6
template <int MU>
__device__ __forceinline__ int lc(int s) { return (s >> (2 * MU)) & 3; }

// shared-memory x: float4 group k holds complex components 2k and 2k+1,
// component c = spin * 3 + colour; row k has 256 sites and one zero "ghost"
// site that hops leaving the domain read instead of a neighbour
constexpr int SX_STRIDE = 264;
constexpr int SX_GHOST = 256;  // 8 zero sites, one per 16-byte bank group
constexpr int SX_BYTES = 6 * SX_STRIDE * 16;
__device__ __forceinline__ void st_load_x(const float4* sx, int site, Spinor<float>& p) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 v = sx[k * SX_STRIDE + site];
    p.v[(2 * k) / 3][(2 * k) % 3] = make_cx(v.x, v.y);
    p.v[(2 * k + 1) / 3][(2 * k + 1) % 3] = make_cx(v.z, v.w);
  }
}

// acc += both intra-domain hops of direction MU (operand x from shared memory).
// x, y, z: a warp holds sites with every coordinate value along MU, so the
// hops are computed for all lanes without branches; a hop that would leave
// the domain reads the zero ghost site (and some valid link) and adds an
// exact zero.  Straight-line code lets the compiler overlap the shared-memory
// loads of several hops.  t: a warp has one t value, the branches are uniform.
// FIRST: this direction's forward hop starts the sum (acc is assigned, not
// added to); only for the branch-free directions
template <int MU, bool HALF, bool FIRST = false>
__device__ __forceinline__ void st_intra(const float4* sx, const unsigned char* sl, int s, Spinor<float>& acc) {
  constexpr int step = 1 << (2 * MU);
  const int c = lc<MU>(s);
  if (MU < 3) {
    {
      Spinor<float> p;
      st_load_x(sx, c < 3 ? s + step : SX_GHOST + ((s + step) & 7), p);
      HalfSpinor<float> h, uh;
      project<MU, -1>(p, h);
      const SU3<float> u = StageT<HALF>::link(sl, MU, s);
      su3_mul(u, h, uh);
      if (FIRST) rebuild<MU, -1>(acc, uh);
      else accumulate<MU, -1>(acc, uh);
    }
    {
      const int nb = c > 0 ? s - step : SX_GHOST + ((s - step) & 7);
      Spinor<float> p;
      st_load_x(sx, nb, p);
      HalfSpinor<float> h, uh;
      project<MU, +1>(p, h);
      const SU3<float> u = StageT<HALF>::link(sl, MU, c > 0 ? s - step : s);
      su3_dag_mul(u, h, uh);
      accumulate<MU, +1>(acc, uh);
    }
    return;
  }
  if (c < 3) {
    Spinor<float> p;
    st_load_x(sx, s + step, p);
    HalfSpinor<float> h, uh;
    project<MU, -1>(p, h);
    const SU3<float> u = StageT<HALF>::link(sl, MU, s);
    su3_mul(u, h, uh);
    accumulate<MU, -1>(acc, uh);
  }
  if (c > 0) {
    Spinor<float> p;
    st_load_x(sx, s - step, p);
    HalfSpinor<float> h, uh;
    project<MU, +1>(p, h);
    const SU3<float> u = StageT<HALF>::link(sl, MU, s - step);
    su3_dag_mul(u, h, uh);
    accumulate<MU, +1>(acc, uh);
  }
}

// Surface term as face tasks.  The hops that enter a 4^4 domain from its
// neighbours end on its eight faces (direction MU, side 0: sites with
// c_MU = 3, forward hop; side 1: c_MU = 0, backward hop), 64 sites each, 512
// per domain.  Thread tau takes face site f = tau & 63 of both sides of
// direction MU = tau >> 6 (two warps per direction, so the branches on MU
// are warp-uniform and no lane idles).  A task's result U P x (a half
// spinor) goes to a slot in shared memory; the site's thread adds the slots
// of its faces afterwards.
// Slots: float4 [MU 4][side 2][3][64] = 24 KB at the start of the x buffer (not
// yet in use; the ghost sites it overlaps are cleared before x is stored).
// The halo has the slots' layout, one block per domain and right-hand side.
__device__ __forceinline__ int face_site(int mu, int side, int f) {
  const int lo = f & ((1 << (2 * mu)) - 1);
  const int hi = f >> (2 * mu);
  return lo | ((side ? 0 : 3) << (2 * mu)) | (hi << (2 * mu + 2));
}
__device__ __forceinline__ int face_index(int mu, int s) {
  const int lo = s & ((1 << (2 * mu)) - 1);
  const int hi = s >> (2 * mu + 2);
  return lo | (hi << (2 * mu));
}
__device__ __forceinline__ float4* face_slot(float4* slots, int mu, int side, int k, int f) {
  return slots + ((mu * 2 + side) * 3 + k) * 64 + f;
}
__device__ __forceinline__ float4* halo_slot(float4* halo, int domr, int mu, int side, int k, int f) {
  return halo + ((size_t)(domr * 8 + mu * 2 + side) * 3 + k) * 64 + f;
}
__device__ __forceinline__ void half_to_f4(const HalfSpinor<float>& h, float4 v[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const cx<float> a0 = h.h[(2 * k) / 3][(2 * k) % 3];
    const cx<float> a1 = h.h[(2 * k + 1) / 3][(2 * k + 1) % 3];
    v[k] = make_float4(a0.re, a0.im, a1.re, a1.im);
  }
}
__device__ __forceinline__ void f4_to_half(const float4 v[3], HalfSpinor<float>& h) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    h.h[(2 * k) / 3][(2 * k) % 3] = make_cx(v[k].x, v[k].y);
    h.h[(2 * k + 1) / 3][(2 * k + 1) % 3] = make_cx(v[k].z, v[k].w);
  }
}

// Producer: after the sweeps, x (in shared memory) is this domain's final
// iterate.  Thread tau handles face site f of both sides of direction MU:
// the side-0 site (c_MU = 3) sends U_MU(m)^dag P+ x(m) to the forward
// neighbour, whose backward hop it is; the side-1 site (c_MU = 0) sends
// P- x(m) to the backward neighbour, whose forward hop it is.  The face index
// f is the same on both ends of a hop.
template <int MU, bool HALF>
__device__ __forceinline__ void st_halo_out_dir(const Geom& g, const float4* sx, const unsigned char* sl,
                                                float4* halo, int dom, int rhs_off, int f) {
  {
    const int m = face_site(MU, 0, f);
    Spinor<float> p;
    st_load_x(sx, m, p);
    HalfSpinor<float> h, uh;
    project<MU, +1>(p, h);
    const SU3<float> u = StageT<HALF>::link(sl, MU, m);
    su3_dag_mul(u, h, uh);
    float4 v[3];
    half_to_f4(uh, v);
    const int nd = __ldg(g.nbr + dom * 8 + 2 * MU) + rhs_off;
#pragma unroll
    for (int k = 0; k < 3; ++k) *halo_slot(halo, nd, MU, 1, k, f) = v[k];
  }
  {
    const int m = face_site(MU, 1, f);
    Spinor<float> p;
    st_load_x(sx, m, p);
    HalfSpinor<float> h;
    project<MU, -1>(p, h);
    float4 v[3];
    half_to_f4(h, v);
    const int nd = __ldg(g.nbr + dom * 8 + 2 * MU + 1) + rhs_off;
#pragma unroll
    for (int k = 0; k < 3; ++k) *halo_slot(halo, nd, MU, 0, k, f) = v[k];
  }
}
template <bool HALF>
__device__ __forceinline__ void st_halo_out(const Geom& g, const float4* sx, const unsigned char* sl, float4* halo,
                                            int dom, int rhs_off, int s) {
  const int f = s & 63;
  switch (s >> 6) {  // warp-uniform
    case 0: st_halo_out_dir<0, HALF>(g, sx, sl, halo, dom, rhs_off, f); break;
    case 1: st_halo_out_dir<1, HALF>(g, sx, sl, halo, dom, rhs_off, f); break;
    case 2: st_halo_out_dir<2, HALF>(g, sx, sl, halo, dom, rhs_off, f); break;
    default: st_halo_out_dir<3, HALF>(g, sx, sl, halo, dom, rhs_off, f); break;
  }
}

// Receiver: the domain's halo block has the layout of the slots and arrives
// there by one bulk copy.  Then, with the links staged, the forward hop's
// P- x is multiplied in place by this domain's U_MU(n); the backward hop's
// U^dag P+ x is complete.  Only t faces can carry the antiperiodic sign.
constexpr int HALO_F4 = 8 * 3 * 64;              // float4 per domain
constexpr unsigned HALO_BYTES = HALO_F4 * 16;    // 24 KB
template <bool HALF>
__device__ __forceinline__ void st_face_tasks(const Geom& g, const unsigned char* sl, int dom, int s, float4* slots) {
  const int mu = s >> 6, f = s & 63;
  float4 v[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) v[k] = *face_slot(slots, mu, 0, k, f);
  HalfSpinor<float> h, uh;
  f4_to_half(v, h);
  const SU3<float> u = StageT<HALF>::link(sl, mu, face_site(mu, 0, f));
  su3_mul(u, h, uh);
  if (mu == 3) {
    const int tf = __ldg(g.tflag + dom);
    if ((tf >> 6) & 1) scale_half(uh, (float)g.bc_t);
    if ((tf >> 7) & 1) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float4* w = face_slot(slots, mu, 1, k, f);
        const float4 t = *w;
        const float sg = (float)g.bc_t;
        *w = make_float4(sg * t.x, sg * t.y, sg * t.z, sg * t.w);
      }
    }
  }
  half_to_f4(uh, v);
#pragma unroll
  for (int k = 0; k < 3; ++k) *face_slot(slots, mu, 0, k, f) = v[k];
}

// acc += the slot of this site's face in direction MU, without branches.  In
// a 4^4 domain a site has at most one face per direction: c_MU = 3 (side 0,
// forward hop, rebuilt with 1 - gamma_MU) or c_MU = 0 (side 1, backward hop,
// 1 + gamma_MU).  The rebuild is written as the side-1 form with the lower
// spins scaled by sg = -1 for side 0 (the two forms differ only there), and
// a site with no face in MU reads some slot and adds it with weight w = 0.
// With w and sg equal to +-1 or 0 every fma is an exact addition.
template <int MU>
__device__ __forceinline__ void st_face_take(const float4* slots, int s, Spinor<float>& acc) {
  const int c = lc<MU>(s);
  const int side = c == 0;
  const float w = (c == 0 || c == 3) ? 1.0f : 0.0f;
  const float sg = side ? w : -w;
  const int f = face_index(MU, s);
  HalfSpinor<float> uh;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 v = *face_slot(const_cast<float4*>(slots), MU, side, k, f);
    uh.h[(2 * k) / 3][(2 * k) % 3] = make_cx(v.x, v.y);
    uh.h[(2 * k + 1) / 3][(2 * k + 1) % 3] = make_cx(v.z, v.w);
  }
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    const cx<float> h0 = uh.h[0][col], h1 = uh.h[1][col];
    acc.v[0][col] = cfma(w, h0, acc.v[0][col]);
    acc.v[1][col] = cfma(w, h1, acc.v[1][col]);
    // spins 2 and 3 of the (1 + gamma_MU) rebuild (accumulate1 with PM = +1)
    if (MU == 0) {
      acc.v[2][col] = cfma(sg, times_i(h1), acc.v[2][col]);
      acc.v[3][col] = cfma(sg, times_i(h0), acc.v[3][col]);
    } else if (MU == 1) {
      acc.v[2][col] = cfma(sg, h1, acc.v[2][col]);
      acc.v[3][col] = cfma(-sg, h0, acc.v[3][col]);
    } else if (MU == 2) {
      acc.v[2][col] = cfma(sg, times_i(h0), acc.v[2][col]);
      acc.v[3][col] = cfma(sg, times_mi(h1), acc.v[3][col]);
    } else {
      acc.v[2][col] = cfma(sg, h0, acc.v[2][col]);
      acc.v[3][col] = cfma(sg, h1, acc.v[3][col]);
    }
  }
}

// the slots of this thread's faces, summed into acc
__device__ __forceinline__ void st_face_sum(const float4* slots, int s, Spinor<float>& acc) {
  st_face_take<0>(slots, s, acc);
  st_face_take<1>(slots, s, acc);
  st_face_take<2>(slots, s, acc);
  st_face_take<3>(slots, s, acc);
}

template <bool HALF>
__device__ __forceinline__ void st_clover(const unsigned char* sc, int s, Spinor<float>& psi) {
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    CloverBlockF32 blk;
    StageT<HALF>::clover_block(sc, s, b, blk);
    cx<float> x[6], y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) x[i] = psi.v[2 * b + i / 3][i % 3];
    herm6_mul<float>(blk, x, y);
#pragma unroll
    for (int i = 0; i < 6; ++i) psi.v[2 * b + i / 3][i % 3] = y[i];
  }
}

__device__ __forceinline__ void st_store_x(float4* sx, int s, const Spinor<float>& a) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const cx<float> a0 = a.v[(2 * k) / 3][(2 * k) % 3];
    const cx<float> a1 = a.v[(2 * k + 1) / 3][(2 * k + 1) % 3];
    sx[k * SX_STRIDE + s] = make_float4(a0.re, a0.im, a1.re, a1.im);
  }
}

// Record a wait that gave up and leave: give the copies one more bounded
// wait each (the decision is uniform across the CTA).
__device__ __forceinline__ void st_give_up(int* status, int tid, bool wait0, uint64_t* bar0, unsigned par0,
                                           bool wait1, uint64_t* bar1, unsigned par1) {
  if (tid == 0) atomicExch(status, QCD_ERR_TIMEOUT);
  if (wait0) mbar_wait_bounded(bar0, par0);
  if (wait1) mbar_wait_bounded(bar1, par1);
}

// What one half-sweep does besides its colour: whether it has a surface term
// (all but the very first), whether it ends with the residual update (all
// but the last sweep), whether it is the first sweep (its input is the
// float32 source s_in32, if that is set) or the last one (the iterate goes
// to x_out32 or x), and whether it writes the neighbours' halo (all but the
// very last).
struct ItemMode {
  int colour, do_surface, do_update, first, last, do_halo;
};

template <bool HALF, typename SIO>
__device__ __forceinline__ ItemMode launch_mode(const StagedArgs<HALF, SIO>& a) {
  return ItemMode{a.colour, a.do_surface, a.do_update, 1, 1, a.do_halo};
}

// Thread 0: initialise the three mbarriers (the CTA's first item only) and
// issue the bulk copies of the domain's links and C_inv.  Before a later
// item's copies overwrite them, the earlier item's generic reads of the
// buffers (ordered by a CTA barrier) are ordered before the async writes.
template <bool HALF, typename SIO>
__device__ __forceinline__ void st_issue_staging(const StagedArgs<HALF, SIO>& a, int dom, int use,
                                                 unsigned char* sl, unsigned char* sc, uint64_t* lbar,
                                                 uint64_t* cbar, uint64_t* hbar) {
  using ST = StageT<HALF>;
  if (use == 0) {
    mbar_init(lbar, 1);
    mbar_init(cbar, 1);
    mbar_init(hbar, 1);
  } else {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  mbar_expect_tx(lbar, ST::LINK_BYTES + a.extra_tx);
  bulk_copy_g2s(sl, a.links + (size_t)dom * ST::LINK_BYTES, ST::LINK_BYTES, lbar);
  mbar_expect_tx(cbar, ST::CLOV_BYTES);
  bulk_copy_g2s(sc, a.clov + (size_t)dom * ST::CLOV_BYTES, ST::CLOV_BYTES, cbar);
}

// One half-sweep of one domain (all of the CTA's right-hand sides).
// HALF: float16 links and C_inv (two CTAs per SM); SIO: storage of s and x.
// SPT: sites per thread.  With SPT = 1 a CTA has 256 threads, one per site;
// with SPT = 2 it has 128 threads, thread tau holding sites tau and
// tau + 128 (the same x, y, z, t and t + 2), which gives each thread two
// independent streams of the same arithmetic.  The arithmetic per site is
// the same in both; the autotuner picks the faster shape.
// use: how many items this CTA ran before (the staging barriers' phase);
// hcount: halo copies this CTA issued before (the halo barrier's phase),
// advanced here; issue: thread 0 issues the staging copies here (else the
// caller did); pdl_wait: wait for the previous grid before reading its
// outputs; flow: the halo was written by other CTAs of this grid (ordered
// by flags), so order those generic writes before the async-proxy copy.
// Returns false if a wait gave up (status set, copies drained).
template <bool HALF, typename SIO, int SPT>
__device__ __forceinline__ bool sap_staged_item(const StagedArgs<HALF, SIO>& a, const ItemMode& m, int blk, int use,
                                                int& hcount, bool issue, bool pdl_wait, bool flow) {
  constexpr int NT = ST_THREADS / SPT;
  extern __shared__ __align__(128) unsigned char smem[];
  using ST = StageT<HALF>;
  float4* sx = reinterpret_cast<float4*>(smem);                              // 24 KB
  unsigned char* sl = smem + SX_BYTES;                                        // links
  unsigned char* sc = sl + ST::LINK_BYTES;                                     // C_inv
  uint64_t* lbar = reinterpret_cast<uint64_t*>(sc + ST::CLOV_BYTES);  // staged links
  uint64_t* cbar = lbar + 1;                                          // staged C_inv
  uint64_t* hbar = lbar + 2;                                          // halo copy
  const Geom& g = a.g;
  const int tid = threadIdx.x;
  const int dom = m.colour * g.nhalf + blk;
  const unsigned spar = use & 1;

  if (issue && tid == 0) st_issue_staging(a, dom, use, sl, sc, lbar, cbar, hbar);
  // the staged links and C_inv are constant during a solve; everything read
  // below may come from the previous launch, which must be complete
  if (pdl_wait) asm volatile("griddepcontrol.wait;" ::: "memory");
  // right-hand sides of this CTA: all of them, or (grid y > 1) the one of blockIdx.y
  const int r_begin = gridDim.y > 1 ? (int)blockIdx.y : 0;
  const int r_end = gridDim.y > 1 ? r_begin + 1 : a.nrhs;
  for (int r = r_begin; r < r_end; ++r) {
    const int i = r - r_begin;  // this CTA's i-th right-hand side
    const int domr = dom + r * g.ndom;  // this right-hand side's copy of the domain
    const int rhs_off = r * g.ndom;
    const unsigned hpar = hcount & 1;
    if (i > 0) __syncthreads();  // every thread is done with the previous rhs's x in shared memory
    if (m.do_surface && tid == 0) {
      // the halo lands in the slots (the start of the x buffer); order the
      // earlier generic accesses to it before the asynchronous copy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (flow) asm volatile("fence.proxy.async.global;" ::: "memory");
      mbar_expect_tx(hbar, HALO_BYTES + a.extra_htx);
      bulk_copy_g2s(sx, a.halo + (size_t)domr * HALO_F4, HALO_BYTES, hbar);
    }
    if (m.do_surface) ++hcount;
    Spinor<float> src[SPT];
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
      if (m.first && a.s_in32.p) a.s_in32.load(g, domr, tid + j * NT, src[j]);
      else a.s_in.load(g, domr, tid + j * NT, src[j]);
    }
    if (i == 0) __syncthreads();  // barrier initialisation visible to every thread
    {
      const bool ok_l = i > 0 || mbar_wait_bounded(lbar, spar);
      const bool ok_h = !m.do_surface || mbar_wait_bounded(hbar, hpar);
      if (__syncthreads_or(!(ok_l && ok_h))) {
        st_give_up(a.status, tid, !ok_l, lbar, spar, !ok_h, hbar, hpar);
        if (i == 0) mbar_wait_bounded(cbar, spar);
        return false;
      }
    }
    Spinor<float> acc[SPT];
    if (m.do_surface) {
#pragma unroll
      for (int j = 0; j < SPT; ++j) st_face_tasks<HALF>(g, sl, dom, tid + j * NT, sx);
      __syncthreads();
#pragma unroll
      for (int j = 0; j < SPT; ++j) {
        zero(acc[j]);
        st_face_sum(sx, tid + j * NT, acc[j]);
      }
      __syncthreads();  // every thread has taken its face slots before x overwrites them
    }
    if (i == 0) {
      // C_inv is first needed here
      const bool ok_c = mbar_wait_bounded(cbar, spar);
      if (__syncthreads_or(!ok_c)) {
        st_give_up(a.status, tid, true, cbar, spar, false, cbar, spar);
        return false;
      }
    }
    if (m.do_surface) {
#pragma unroll
      for (int j = 0; j < SPT; ++j) {
        st_clover<HALF>(sc, tid + j * NT, acc[j]);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            src[j].v[sp][c].re = fmaf(a.kappa, acc[j].v[sp][c].re, src[j].v[sp][c].re);
            src[j].v[sp][c].im = fmaf(a.kappa, acc[j].v[sp][c].im, src[j].v[sp][c].im);
          }
      }
    }
    if (tid < 48) sx[(tid >> 3) * SX_STRIDE + SX_GHOST + (tid & 7)] = make_float4(0.f, 0.f, 0.f, 0.f);  // face slots overlap it
#pragma unroll
    for (int j = 0; j < SPT; ++j) st_store_x(sx, tid + j * NT, src[j]);
    __syncthreads();

    Spinor<float> xk[SPT];
#pragma unroll
    for (int j = 0; j < SPT; ++j) xk[j] = src[j];
    const int napp = a.n_jac + (m.do_update ? 1 : 0);
    for (int it = 0; it < napp; ++it) {
      // the x hops start the sum (no zeroing); the t hops' warp-uniform
      // branches follow, then one straight-line stretch (y, z hops and the
      // clover multiply)
#pragma unroll
      for (int j = 0; j < SPT; ++j) {
        const int s = tid + j * NT;
        st_intra<0, HALF, true>(sx, sl, s, acc[j]);
        st_intra<3, HALF>(sx, sl, s, acc[j]);
        st_intra<1, HALF>(sx, sl, s, acc[j]);
        st_intra<2, HALF>(sx, sl, s, acc[j]);
        st_clover<HALF>(sc, s, acc[j]);
      }
      if (it < a.n_jac) {
#pragma unroll
        for (int j = 0; j < SPT; ++j)
#pragma unroll
          for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              xk[j].v[sp][c].re = fmaf(a.kappa, acc[j].v[sp][c].re, src[j].v[sp][c].re);
              xk[j].v[sp][c].im = fmaf(a.kappa, acc[j].v[sp][c].im, src[j].v[sp][c].im);
            }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < SPT; ++j) st_store_x(sx, tid + j * NT, xk[j]);
        __syncthreads();
      } else {
#pragma unroll
        for (int j = 0; j < SPT; ++j) {
          const int s = tid + j * NT;
          Spinor<float> b;
          a.b.load(g, domr, s, b);
#pragma unroll
          for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float re = src[j].v[sp][c].re + b.v[sp][c].re - xk[j].v[sp][c].re;
              const float im = src[j].v[sp][c].im + b.v[sp][c].im - xk[j].v[sp][c].im;
              acc[j].v[sp][c].re = fmaf(a.kappa, acc[j].v[sp][c].re, re);
              acc[j].v[sp][c].im = fmaf(a.kappa, acc[j].v[sp][c].im, im);
            }
          a.s_out.store(g, domr, s, acc[j]);
        }
      }
    }
    if (m.do_halo) {  // sx holds the final iterate
#pragma unroll
      for (int j = 0; j < SPT; ++j) st_halo_out<HALF>(g, sx, sl, a.halo, dom, rhs_off, tid + j * NT);
    }
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
      if (m.last && a.x_store) a.x.store(g, domr, tid + j * NT, xk[j]);
      if (m.last && a.x_out32.p) a.x_out32.store(g, domr, tid + j * NT, xk[j]);
    }
  }
  return true;
}

// one launch = one half-sweep: the launch's mode and the CTA's domain
template <bool HALF, typename SIO, int SPT>
__device__ __forceinline__ void sap_staged_body(const StagedArgs<HALF, SIO>& a, int blk) {
  if (loop_idle(a.g) || (a.skip && *(volatile const int*)a.skip)) return;
  // programmatic dependent launch: the next launch in the stream may start
  // its CTAs while this grid drains
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  int hcount = 0;
  sap_staged_item<HALF, SIO, SPT>(a, launch_mode(a), blk, 0, hcount, true, true, false);
}

template <bool HALF, typename SIO, int SPT>
__global__ void __launch_bounds__(ST_THREADS / SPT, HALF ? 2 : 1) sap_staged_kernel(StagedArgs<HALF, SIO> a) {
  sap_staged_body<HALF, SIO, SPT>(a, blockIdx.x);
}

// ---------------------------------------------------------------------------
// M_SAP in one launch: half-sweeps ordered by per-domain flags
// ---------------------------------------------------------------------------
// A grid of resident CTAs takes the work items of a whole M_SAP in order
// from a ticket counter: item j is half-sweep k = j / nhalf (sweep k / 2,
// colour k % 2) of the colour's domain j % nhalf.  Item (k, d) reads the
// halo that its eight neighbours (the other colour) wrote in half-sweep
// k - 1, and the s that its own domain wrote in half-sweep k - 2, which
// those neighbours' half-sweep k - 1 waited for.  So it waits for the eight
// neighbours' flags to reach k, and a finished item sets its domain's flag
// to k + 1 (release after its global writes; the waits acquire).  Its halo
// writes go to the neighbours' blocks, whose previous readers (their
// half-sweep k - 1) are among the items it waited for.  Every item depends
// only on items with smaller tickets, which CTAs that are running hold, so
// the order cannot deadlock.  Compared with one launch per half-sweep, no
// CTA waits for a whole grid to drain, and the CTAs' staging copies spread
// over time instead of coming in bursts at the start of every wave.
// The last CTA to leave clears the flags and the counters for the next use.
struct FlowArgs {
  int* flags;      // [domain]: half-sweeps finished + 1 of its last item (0 at rest)
  int* ctr;        // [0] ticket, [1] CTAs retired
  int n_sap;
  int stagger_ns;  // the second half of the CTAs start this much later
};

// Bounded acquire-wait for *flag >= need.  Gives up after 2^22 polls or
// half a second, or as soon as another CTA has reported a failure.
__device__ __forceinline__ bool flow_wait(const int* flag, int need, const int* status) {
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < (1 << 22); ++i) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
    if (v >= need) return true;
    if ((i & 31) == 31) {
      if (*(volatile const int*)status != 0) return false;
      if (global_ns() - t0 > 500000000ull) return false;
    }
    __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Each CTA holds the ticket after the one it runs, so that, while an item
// computes, the next item's links and C_inv are already on their way to L2.
// A finished item's flag is released only after the next item's staging
// copies are issued (the release waits for the item's writes), and always
// before the CTA waits on any flag, so no CTA waits while holding an
// unreleased flag.  Holding the next ticket cannot block anyone for ever:
// the item in hand depends only on smaller tickets.
template <bool HALF, typename SIO>
__global__ void __launch_bounds__(ST_THREADS, HALF ? 2 : 1) sap_flow_kernel(StagedArgs<HALF, SIO> a, FlowArgs f) {
  extern __shared__ __align__(128) unsigned char smem[];
  using ST = StageT<HALF>;
  unsigned char* sl = smem + SX_BYTES;
  unsigned char* sc = sl + ST::LINK_BYTES;
  uint64_t* lbar = reinterpret_cast<uint64_t*>(sc + ST::CLOV_BYTES);
  __shared__ int s_item, s_next, s_last;
  const Geom& g = a.g;
  if (loop_idle(g) || (a.skip && *(volatile const int*)a.skip)) return;  // the same for every CTA
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // The counters and flags belong to the previous use until its grid has
  // completed, and the earlier launches' outputs are read below: wait for
  // the previous grid (which itself waited for its own predecessor) first.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int tid = threadIdx.x;
  const int nhalf = g.nhalf;
  const int total = 2 * (f.n_sap + 1) * nhalf;
  if (f.stagger_ns > 0 && blockIdx.x >= gridDim.x / 2 && tid == 0) {
    const unsigned long long t0 = global_ns();
    for (int i = 0; i < 4096 && global_ns() - t0 < (unsigned long long)f.stagger_ns; ++i) __nanosleep(256);
  }
  if (tid == 0) {
    s_item = atomicAdd(f.ctr, 1);
    s_next = atomicAdd(f.ctr, 1);
  }
  __syncthreads();
  int j = s_item, jn = s_next;
  int use = 0, hcount = 0;
  int pending = -1, pending_val = 0;  // (thread 0) finished item whose flag is not yet released
  auto release = [&]() {
    if (pending >= 0) {
      __threadfence();
      asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(f.flags + pending), "r"(pending_val) : "memory");
      pending = -1;
    }
  };
  while (j < total) {
    const int k = j / nhalf, blk = j - k * nhalf;
    const int sweep = k >> 1, colour = k & 1;
    const ItemMode m{colour, k > 0, sweep < f.n_sap, sweep == 0, sweep == f.n_sap,
                     !(sweep == f.n_sap && colour == 1)};
    const int dom = colour * nhalf + blk;
    if (tid == 0) {
      // the staging copies need nothing from other items: issue them first
      st_issue_staging(a, dom, use, sl, sc, lbar, lbar + 1, lbar + 2);
      if (jn < total) {
        const int kn = jn / nhalf;
        const int domn = (kn & 1) * nhalf + (jn - kn * nhalf);
        prefetch_l2(a.links + (size_t)domn * ST::LINK_BYTES, ST::LINK_BYTES);
        prefetch_l2(a.clov + (size_t)domn * ST::CLOV_BYTES, ST::CLOV_BYTES);
      }
      release();
    }
    if (k > 0) {
      // warp 1 waits for the neighbours while warp 0 releases
      bool ok = true;
      if (tid >= 32 && tid < 40) ok = flow_wait(f.flags + __ldg(g.nbr + dom * 8 + (tid - 32)), k, a.status);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicExch(a.status, QCD_ERR_TIMEOUT);
        mbar_wait_bounded(lbar, use & 1);
        mbar_wait_bounded(lbar + 1, use & 1);
        break;
      }
    }
    if (!sap_staged_item<HALF, SIO, 1>(a, m, blk, use, hcount, false, false, true)) break;
    __syncthreads();  // the item's global writes are done and its shared memory is free
    if (tid == 0) {
      pending = dom;
      pending_val = k + 1;
      s_item = jn;
      s_next = (jn >= total || *(volatile const int*)a.status != 0) ? total : atomicAdd(f.ctr, 1);
    }
    __syncthreads();
    j = s_item;
    jn = s_next;
    ++use;
  }
  __syncthreads();
  if (tid == 0) {
    release();
    __threadfence();
    s_last = atomicAdd(f.ctr + 1, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    for (int d = tid; d < g.ndom; d += blockDim.x) f.flags[d] = 0;
    if (tid == 0) {
      f.ctr[0] = 0;
      f.ctr[1] = 0;
    }
  }
}

// Ragged batch: one launch covers one half-sweep of every lattice.  Block b
// belongs to lattice block_lat[b] and is its domain b - block_first[lat];
// the block copies that lattice's arguments (geometry, kappa, field and
// staging pointers) to shared memory first.  Every lattice must have 4^4
// domains.
template <bool HALF, typename SIO>
__global__ void __launch_bounds__(ST_THREADS, HALF ? 2 : 1)
    sap_staged_batch_kernel(const StagedArgs<HALF, SIO>* __restrict__ tab, const int* __restrict__ block_lat,
                            const int* __restrict__ block_first) {
  __shared__ StagedArgs<HALF, SIO> sa;
  const int lat = __ldg(block_lat + blockIdx.x);
  {
    const int* src = reinterpret_cast<const int*>(tab + lat);
    int* dst = reinterpret_cast<int*>(&sa);
    for (int k = threadIdx.x; k < (int)(sizeof(sa) / sizeof(int)); k += blockDim.x) dst[k] = __ldg(src + k);
  }
  __syncthreads();
  sap_staged_body<HALF, SIO, 1>(sa, (int)blockIdx.x - __ldg(block_first + lat));
}

// ---------------------------------------------------------------------------
// staging layouts, built from the internal layouts
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
    l16[((size_t)(dom * 4 + mu) * 256 + s) * L16_H2 + e] = __floats2half2_rn((float)v.x, (float)v.y);
    l32[o] = make_float2((float)v.x, (float)v.y);
  }
  l16[((size_t)(dom * 4 + mu) * 256 + s) * L16_H2 + 9] = __floats2half2_rn(0.f, 0.f);
}

__global__ void build_clover_stage_kernel(Geom g, const double2* c64, uint4* c16, float4* c32) {
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gid >= g.vol) return;
  const int s = (int)(gid & 255);
  const int dom = (int)(gid >> 8);
  __half2* h = reinterpret_cast<__half2*>(c16 + (size_t)(dom * 256 + s) * C16_U4);
  float* f = reinterpret_cast<float*>(c32 + (size_t)(dom * 256 + s) * C32_F4);
  for (int b = 0; b < 2; ++b) {
    for (int k = 0; k < 18; ++k) {
      const double2 v = c64[(((size_t)(dom * 36 + 18 * b + k)) << 8) + s];
      h[18 * b + k] = __floats2half2_rn((float)v.x, (float)v.y);
      f[36 * b + 2 * k] = (float)v.x;
      f[36 * b + 2 * k + 1] = (float)v.y;
    }
  }
  for (int k = 72; k < 76; ++k) f[k] = 0.f;
}

bool sap_staged_available(const qcd_ctx* ctx) {
  const Geom& g = ctx->geom;
  return g.d[0] == 4 && g.d[1] == 4 && g.d[2] == 4 && g.d[3] == 4 && ctx->st_link16 && ctx->st_clov16;
}

// x buffer, staged links and C_inv, three mbarriers
template <bool HALF>
constexpr int st_smem_bytes() {
  return SX_BYTES + StageT<HALF>::LINK_BYTES + StageT<HALF>::CLOV_BYTES + 32;
}

void build_sap_staging(qcd_ctx* ctx, cudaStream_t st) {
  const Geom& g = ctx->geom;
  if (!(g.d[0] == 4 && g.d[1] == 4 && g.d[2] == 4 && g.d[3] == 4)) return;
  const size_t nd = (size_t)g.ndom;
  if (!ctx->st_link16) {
    QCD_CUDA_CHECK(cudaMalloc(&ctx->st_link16, nd * StageT<true>::LINK_BYTES));
    QCD_CUDA_CHECK(cudaMalloc(&ctx->st_link32, nd * StageT<false>::LINK_BYTES));
    QCD_CUDA_CHECK(cudaMalloc(&ctx->st_clov16, nd * StageT<true>::CLOV_BYTES));
    QCD_CUDA_CHECK(cudaMalloc(&ctx->st_clov32, nd * StageT<false>::CLOV_BYTES));
    const int s16 = st_smem_bytes<true>();
    const int s32 = st_smem_bytes<false>();
    QCD_CUDA_CHECK(cudaFuncSetAttribute(sap_staged_kernel<true, F16Spinor, 1>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, s16));
    QCD_CUDA_CHECK(cudaFuncSetAttribute(sap_staged_kernel<true, F16Spinor, 2>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, s16));
    QCD_CUDA_CHECK(cudaFuncSetAttribute(sap_staged_kernel<true, F32Spinor, 1>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, s16));
    QCD_CUDA_CHECK(cudaFuncSetAttribute(sap_staged_kernel<true, F32Spinor, 2>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, s16));
    QCD_CUDA_CHECK(cudaFuncSetAttribute(sap_staged_kernel<false, F32Spinor, 1>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, s32));
    QCD_CUDA_CHECK(cudaFuncSetAttribute(sap_staged_kernel<false, F32Spinor, 2>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, s32));
    QCD_CUDA_CHECK(cudaFuncSetAttribute(sap_flow_kernel<true, F16Spinor>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, s16));
    QCD_CUDA_CHECK(cudaFuncSetAttribute(sap_flow_kernel<true, F32Spinor>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, s16));
    QCD_CUDA_CHECK(cudaFuncSetAttribute(sap_flow_kernel<false, F32Spinor>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, s32));
    QCD_CUDA_CHECK(cudaMalloc(&ctx->flow_state, sizeof(int) * (2 + nd)));
    QCD_CUDA_CHECK(cudaMemset(ctx->flow_state, 0, sizeof(int) * (2 + nd)));
  }
  LaunchScope ls(ctx, QCD_KC_OTHER, st);
  build_link_stage_kernel<<<grid_for(g.vol * 4, 256), 256, 0, st>>>(g, ctx->u64, (__half2*)ctx->st_link16,
                                                                    (float2*)ctx->st_link32);
  build_clover_stage_kernel<<<grid_for(g.vol, 256), 256, 0, st>>>(g, ctx->cinv64,
                                                                  (uint4*)ctx->st_clov16, (float4*)ctx->st_clov32);
  check_launch();
}

// Algorithm 1 as 2 (n_sap + 1) launches.  s_first_in32 (float32) is the
// first sweep's input, the source itself.  The final iterate goes to x_out32
// if it is set, else to x.  halo holds 96 bytes per site and right-hand side.
template <bool HALF, typename SIO, int SPT>
static void staged_sequence_shape(qcd_ctx* ctx, F32Spinor s_first_in32, SIO s, SIO x, F32Spinor b,
                                  F32Spinor x_out32, float4* halo, int nrhs, int n_sap, int n_jac, cudaStream_t st,
                                  bool rhs_grid = false) {
  StagedArgs<HALF, SIO> a;
  a.g = ctx->geom;
  a.nrhs = nrhs;
  a.n_jac = n_jac;
  a.kappa = (float)ctx->kappa;
  a.b = b;
  a.x = x;
  a.s_out = s;
  a.s_in = s;
  a.halo = halo;
  a.links = (const unsigned char*)(HALF ? ctx->st_link16 : ctx->st_link32);
  a.clov = (const unsigned char*)(HALF ? ctx->st_clov16 : ctx->st_clov32);
  a.status = ctx->d_status;
  // test hook: wait for 16 bytes that no copy brings, so that the bounded
  // wait gives up and reports QCD_ERR_TIMEOUT
  a.extra_tx = ctx->inject == QCD_INJECT_STAGING_WAIT ? 16 : 0;
  a.extra_htx = ctx->inject == QCD_INJECT_HALO_WAIT ? 16 : 0;
  a.skip = nullptr;
  for (int sweep = 0; sweep <= n_sap; ++sweep) {
    a.s_in32 = sweep == 0 ? s_first_in32 : F32Spinor{nullptr};
    a.do_update = sweep == n_sap ? 0 : 1;
    for (int colour = 0; colour < 2; ++colour) {
      a.colour = colour;
      a.do_surface = (sweep == 0 && colour == 0) ? 0 : 1;
      const bool last = sweep == n_sap;
      a.x_out32 = last ? x_out32 : F32Spinor{nullptr};
      a.x_store = (last && !x_out32.p) ? 1 : 0;
      a.do_halo = (last && colour == 1) ? 0 : 1;
      LaunchScope ls(ctx, QCD_KC_SAP_BLOCK, st);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(ctx->geom.nhalf, rhs_grid ? nrhs : 1);
      cfg.blockDim = dim3(ST_THREADS / SPT);
      cfg.dynamicSmemBytes = st_smem_bytes<HALF>();
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      QCD_CUDA_CHECK(cudaLaunchKernelEx(&cfg, sap_staged_kernel<HALF, SIO, SPT>, a));
      check_launch();
    }
  }
}

// Algorithm 1 as one launch of resident CTAs (sap_flow_kernel).
template <bool HALF, typename SIO>
static void flow_sequence(qcd_ctx* ctx, F32Spinor s_first_in32, SIO s, SIO x, F32Spinor b, F32Spinor x_out32,
                          float4* halo, int nrhs, int n_sap, int n_jac, cudaStream_t st, int stagger_ns) {
  QCD_REQUIRE(n_sap >= 1 && 2 * (n_sap + 1) * (long long)ctx->geom.nhalf < (1LL << 31) && n_sap < (1 << 20),
              QCD_ERR_ARG, "one-launch SAP: n_sap out of range");
  StagedArgs<HALF, SIO> a;
  a.g = ctx->geom;
  a.colour = 0;
  a.n_jac = n_jac;
  a.do_surface = a.do_update = a.do_halo = 0;  // per item
  a.nrhs = nrhs;
  a.kappa = (float)ctx->kappa;
  a.s_in = s;
  a.s_out = s;
  a.x = x;
  a.b = b;
  a.s_in32 = s_first_in32;
  a.x_out32 = x_out32;
  a.x_store = x_out32.p ? 0 : 1;
  a.halo = halo;
  a.links = (const unsigned char*)(HALF ? ctx->st_link16 : ctx->st_link32);
  a.clov = (const unsigned char*)(HALF ? ctx->st_clov16 : ctx->st_clov32);
  a.status = ctx->d_status;
  a.extra_tx = ctx->inject == QCD_INJECT_STAGING_WAIT ? 16 : 0;
  a.extra_htx = ctx->inject == QCD_INJECT_HALO_WAIT ? 16 : 0;
  a.skip = nullptr;
  FlowArgs f;
  f.flags = ctx->flow_state + 2;
  f.ctr = ctx->flow_state;
  f.n_sap = n_sap;
  f.stagger_ns = stagger_ns;
  // as many CTAs as can be resident at once (computed once; the batch
  // solve's host threads may get here together)
  static const int resident = [] {
    int dev = 0, sms = 0, per_sm = 0;
    QCD_CUDA_CHECK(cudaGetDevice(&dev));
    QCD_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    QCD_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sap_flow_kernel<HALF, SIO>, ST_THREADS,
                                                                 st_smem_bytes<HALF>()));
    return per_sm * sms;
  }();
  const int total = 2 * (n_sap + 1) * ctx->geom.nhalf;
  const int grid = std::max(1, std::min(total, resident));
  LaunchScope ls(ctx, QCD_KC_SAP_BLOCK, st);
  launch_pdl(sap_flow_kernel<HALF, SIO>, dim3(grid), dim3(ST_THREADS), st_smem_bytes<HALF>(), st, a, f);
  check_launch();
}

// The block-kernel shape is chosen by the autotuner on the first M_SAP of
// each precision, lattice, right-hand-side count and n_jac: it times the
// whole sequence in every shape on the caller's buffers (M_SAP is a function
// of its input alone, so the repeated runs leave the same result) and keeps
// the fastest.  Shapes: one or two sites per thread, and, with several
// right-hand sides, one CTA per domain and right-hand side (each stages the
// domain's links and C_inv for itself; more CTAs where a lattice has too few
// domains to fill the GPU) instead of one CTA running all of them through
// its staged operator.  qcd_set_sap_shape fixes the shape.
// The last two shapes run the whole of M_SAP in one launch (sap_flow_kernel),
// the second of them with half of its CTAs starting later, so that the
// CTAs on one SM load their operators at different times.
static const char* const kSapShapes[] = {"256x1site", "128x2sites", "256x1site_rhs_grid", "one_launch",
                                         "one_launch_staggered"};
constexpr int kFlowStaggerNs = 10000;

template <bool HALF, typename SIO>
static void staged_sequence(qcd_ctx* ctx, F32Spinor s_first_in32, SIO s, SIO x, F32Spinor b, F32Spinor x_out32,
                            float4* halo, int nrhs, int n_sap, int n_jac, cudaStream_t st) {
  auto run = [&](int v) {
    if (v == 1)
      staged_sequence_shape<HALF, SIO, 2>(ctx, s_first_in32, s, x, b, x_out32, halo, nrhs, n_sap, n_jac, st);
    else if (v >= 3 && n_sap >= 1)
      flow_sequence<HALF, SIO>(ctx, s_first_in32, s, x, b, x_out32, halo, nrhs, n_sap, n_jac, st,
                               v == 4 ? kFlowStaggerNs : 0);
    else
      staged_sequence_shape<HALF, SIO, 1>(ctx, s_first_in32, s, x, b, x_out32, halo, nrhs, n_sap, n_jac, st,
                                          v == 2 && nrhs > 1);
  };
  int v = ctx->sap_shape;
  if (v < 0) {
    const Geom& g = ctx->geom;
    char key[128];
    std::snprintf(key, sizeof key, "sap_staged_%s L%dx%dx%dx%d nrhs%d n_sap%d n_jac%d",
                  HALF ? (std::is_same<SIO, F16Spinor>::value ? "f16" : "f16gauge") : "f32", g.L[0], g.L[1], g.L[2],
                  g.L[3], nrhs, n_sap, n_jac);
    // candidates: both thread shapes, the right-hand-side grid (several
    // right-hand sides only) and, with n_sap >= 1, the two one-launch forms
    static const int with_rhs[] = {0, 1, 2, 3, 4}, one_rhs[] = {0, 1, 3, 4};
    const int* cand = nrhs > 1 ? with_rhs : one_rhs;
    const int nc = (nrhs > 1 ? 3 : 2) + (n_sap >= 1 ? 2 : 0);
    const char* names[5];
    for (int c = 0; c < nc; ++c) names[c] = kSapShapes[cand[c]];
    v = cand[tune_pick(ctx, key, nc, names, [&](int c) { run(cand[c]); }, st)];
  }
  run(v);
}

void sap_staged_sequence_f32(qcd_ctx* ctx, F32Spinor s_first_in, F32Spinor s, F32Spinor x, F32Spinor b,
                             float4* halo, int nrhs, int n_sap, int n_jac, cudaStream_t st) {
  staged_sequence<false, F32Spinor>(ctx, s_first_in, s, x, b, F32Spinor{nullptr}, halo, nrhs, n_sap, n_jac, st);
}
void sap_staged_sequence_f16(qcd_ctx* ctx, F32Spinor s_first_in, F16Spinor s, F32Spinor b, F32Spinor x_out,
                             float4* halo, int nrhs, int n_sap, int n_jac, cudaStream_t st) {
  staged_sequence<true, F16Spinor>(ctx, s_first_in, s, F16Spinor{nullptr, nullptr}, b, x_out, halo, nrhs, n_sap, n_jac,
                                   st);
}
void sap_staged_sequence_h16g(qcd_ctx* ctx, F32Spinor s_first_in, F32Spinor s, F32Spinor x, F32Spinor b,
                              float4* halo, int nrhs, int n_sap, int n_jac, cudaStream_t st) {
  staged_sequence<true, F32Spinor>(ctx, s_first_in, s, x, b, F32Spinor{nullptr}, halo, nrhs, n_sap, n_jac, st);
}

// ---------------------------------------------------------------------------
// ragged batch of lattices: M_SAP of every lattice in shared launches
// ---------------------------------------------------------------------------
struct SapBatchPlan {
  int prec = 0;
  int nlat = 0, nlaunch = 0;
  int blocks = 0;                 // domains of one colour, summed over the lattices
  void* d_tab = nullptr;          // StagedArgs [launch][lattice]
  int* d_block_lat = nullptr;     // lattice of every block
  int* d_block_first = nullptr;   // first block of every lattice
};

template <bool HALF, typename SIO>
static void* sap_batch_table(const std::vector<SapLat>& L, int n_sap, int n_jac, int* status, const int* run_flag) {
  static_assert(sizeof(StagedArgs<HALF, SIO>) % sizeof(int) == 0, "argument block is copied as ints");
  const int n = (int)L.size(), nlaunch = 2 * (n_sap + 1);
  std::vector<StagedArgs<HALF, SIO>> h((size_t)nlaunch * n);
  for (int i = 0; i < n; ++i) {
    const qcd_ctx* c = L[i].ctx;
    StagedArgs<HALF, SIO> a;
    std::memset(&a, 0, sizeof a);
    a.g = c->geom;
    a.g.run_flag = run_flag;
    a.nrhs = 1;
    a.n_jac = n_jac;
    a.kappa = (float)c->kappa;
    a.b = L[i].in;
    a.halo = L[i].halo;
    a.links = (const unsigned char*)(HALF ? c->st_link16 : c->st_link32);
    a.clov = (const unsigned char*)(HALF ? c->st_clov16 : c->st_clov32);
    a.status = status;
    a.skip = L[i].skip;
    SIO sv;
    if constexpr (std::is_same<SIO, F16Spinor>::value) sv = F16Spinor{L[i].s16, L[i].s16n};
    else sv = F32Spinor{L[i].s32};
    a.s_in = sv;
    a.s_out = sv;
    int k = 0;
    for (int sweep = 0; sweep <= n_sap; ++sweep) {
      const bool last = sweep == n_sap;
      for (int colour = 0; colour < 2; ++colour, ++k) {
        a.s_in32 = sweep == 0 ? L[i].in : F32Spinor{nullptr};
        a.do_update = last ? 0 : 1;
        a.colour = colour;
        a.do_surface = (sweep == 0 && colour == 0) ? 0 : 1;
        a.do_halo = (last && colour == 1) ? 0 : 1;
        if constexpr (std::is_same<SIO, F16Spinor>::value) {
          a.x = F16Spinor{nullptr, nullptr};
          a.x_out32 = last ? L[i].out : F32Spinor{nullptr};
          a.x_store = 0;
        } else {
          a.x = L[i].out;
          a.x_out32 = F32Spinor{nullptr};
          a.x_store = last ? 1 : 0;
        }
        h[(size_t)k * n + i] = a;
      }
    }
  }
  void* d = nullptr;
  QCD_CUDA_CHECK(cudaMalloc(&d, sizeof(StagedArgs<HALF, SIO>) * h.size()));
  QCD_CUDA_CHECK(cudaMemcpy(d, h.data(), sizeof(StagedArgs<HALF, SIO>) * h.size(), cudaMemcpyHostToDevice));
  QCD_CUDA_CHECK(cudaFuncSetAttribute(sap_staged_batch_kernel<HALF, SIO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      st_smem_bytes<HALF>()));
  return d;
}

SapBatchPlan* sap_batch_plan(const std::vector<SapLat>& L, int sap_prec, int n_sap, int n_jac, int* status,
                             const int* run_flag) {
  for (const SapLat& l : L)
    QCD_REQUIRE(sap_staged_available(l.ctx), QCD_ERR_ARG, "batched SAP: every lattice needs 4^4 domains");
  SapBatchPlan* P = new SapBatchPlan();
  try {
    P->prec = sap_prec;
    P->nlat = (int)L.size();
    P->nlaunch = 2 * (n_sap + 1);
    std::vector<int> lat, first;
    for (int i = 0; i < P->nlat; ++i) {
      first.push_back((int)lat.size());
      for (int d = 0; d < L[i].ctx->geom.nhalf; ++d) lat.push_back(i);
    }
    P->blocks = (int)lat.size();
    QCD_CUDA_CHECK(cudaMalloc(&P->d_block_lat, sizeof(int) * lat.size()));
    QCD_CUDA_CHECK(cudaMemcpy(P->d_block_lat, lat.data(), sizeof(int) * lat.size(), cudaMemcpyHostToDevice));
    QCD_CUDA_CHECK(cudaMalloc(&P->d_block_first, sizeof(int) * first.size()));
    QCD_CUDA_CHECK(cudaMemcpy(P->d_block_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice));
    if (sap_prec == QCD_PREC_HALF) P->d_tab = sap_batch_table<true, F16Spinor>(L, n_sap, n_jac, status, run_flag);
    else if (sap_prec == QCD_PREC_HALF_GAUGE)
      P->d_tab = sap_batch_table<true, F32Spinor>(L, n_sap, n_jac, status, run_flag);
    else P->d_tab = sap_batch_table<false, F32Spinor>(L, n_sap, n_jac, status, run_flag);
  } catch (...) {
    sap_batch_free(P);
    throw;
  }
  return P;
}

void sap_batch_free(SapBatchPlan* P) {
  if (!P) return;
  if (P->d_tab) cudaFree(P->d_tab);
  if (P->d_block_lat) cudaFree(P->d_block_lat);
  if (P->d_block_first) cudaFree(P->d_block_first);
  delete P;
}

template <bool HALF, typename SIO>
static void sap_batch_launches(const SapBatchPlan* P, qcd_ctx* count_ctx, cudaStream_t st) {
  const StagedArgs<HALF, SIO>* tab = static_cast<const StagedArgs<HALF, SIO>*>(P->d_tab);
  for (int k = 0; k < P->nlaunch; ++k) {
    LaunchScope ls(count_ctx, QCD_KC_SAP_BLOCK, st);
    launch_pdl(sap_staged_batch_kernel<HALF, SIO>, dim3(P->blocks), dim3(ST_THREADS), st_smem_bytes<HALF>(), st,
               tab + (size_t)k * P->nlat, (const int*)P->d_block_lat, (const int*)P->d_block_first);
    check_launch();
  }
}

void sap_batch_run(const SapBatchPlan* P, qcd_ctx* count_ctx, cudaStream_t st) {
  if (P->prec == QCD_PREC_HALF) sap_batch_launches<true, F16Spinor>(P, count_ctx, st);
  else if (P->prec == QCD_PREC_HALF_GAUGE) sap_batch_launches<true, F32Spinor>(P, count_ctx, st);
  else sap_batch_launches<false, F32Spinor>(P, count_ctx, st);
}

}  // namespace qcd
