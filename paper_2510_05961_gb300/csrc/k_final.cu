// k_final.cu -- outputs of the MSM evaluation (Sec. 2, Eq. U_contributions;
// Sec. 3.2.2 for the derivatives):
//   phi_i = phi0_i + phi^(1+)_i  (= dE/dq_i),
//   field_i = -grad phi(r_i) (both parts), F_i = q_i field_i,
//   E = 1/2 sum_i q_i phi_i   (each product exact as hi + lo in FP32, summed as
//                              hi + lo pairs by error-free transformations in
//                              a fixed order, FP64 for the final value),
//   W = W0 + W^(1+)           (FP64, fixed-order sums of the block partials),
// written back in the caller's atom order by gathers through the inverse sort
// permutation.
#include "msm_internal.h"

namespace msm {

// Knuth's TwoSum: s + t = a + b exactly (round-to-nearest, no contraction)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a += b for sums kept as hi + lo: the hi parts by TwoSum, every rounding
// error of theirs collected in lo
__device__ __forceinline__ void add_hl(float2& a, float2 b) {
  float s, t;
  two_sum(a.x, b.x, s, t);
  a.x = s;
  a.y = __fadd_rn(a.y, __fadd_rn(b.y, t));
}

__device__ __forceinline__ float2 shfl_down_hl(float2 v, int o) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, o), __shfl_down_sync(0xffffffffu, v.y, o));
}

// The energy sum sum_i q_i phi_i: each product is split exactly as hi + lo
// (lo by FMA) and the terms are summed as hi + lo pairs in a fixed order (warp
// shuffles, then the block, then k_energy over the blocks in order): the
// result is the exact sum up to the FP32 rounding of the lo parts, about
// 2^-47 of sum |q phi|, with no FP64 arithmetic (slow on this GPU) before the
// final conversion; 1/2 is applied at the end (exact).
// The per-atom results go to res in the sorted order (coalesced); k_outputs
// and k_backward_scale_res then gather them into the caller's order, so that their
// stores are coalesced and only one 16-byte load per atom is scattered.
__global__ void __launch_bounds__(kChunk) k_finalize(const SysDev* __restrict__ sys,
                                                     const AtomItem* __restrict__ items, const float4* __restrict__ xq,
                                                     const float* __restrict__ phi_sr, const float* __restrict__ phi_lr,
                                                     const float4* __restrict__ f_sr, const float4* __restrict__ f_lr,
                                                     bool forces, float4* __restrict__ res,
                                                     float2* __restrict__ part_e, float2* __restrict__ part_q) {
  __shared__ float2 red[kChunk / 32][2];
  AtomItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  int local = it.start + threadIdx.x;
  float2 e = make_float2(0.f, 0.f);
  float qs = 0.f, qa = 0.f;  // sum q and sum |q| (FP32: only compared with a 1e-5 threshold)
  if ((int)threadIdx.x < it.count && local < S.n) {
    const int k = S.atom_off + local;
    const float qk = xq[k].w;
    const float ph = phi_sr[k] + phi_lr[k];
    e.x = __fmul_rn(qk, ph);
    e.y = fmaf(qk, ph, -e.x);
    qs = qk;
    qa = fabsf(qk);
    float4 r = make_float4(ph, 0.f, 0.f, 0.f);
    if (forces) {
      const float4 a = f_sr[k], b = f_lr[k];
      r.y = qk * (a.x + b.x);
      r.z = qk * (a.y + b.y);
      r.w = qk * (a.z + b.z);
    }
    res[k] = r;
  }
  for (int o = 16; o > 0; o >>= 1) {
    add_hl(e, shfl_down_hl(e, o));
    qs += __shfl_down_sync(0xffffffffu, qs, o);
    qa += __shfl_down_sync(0xffffffffu, qa, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = e;
    red[threadIdx.x >> 5][1] = make_float2(qs, qa);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 t = red[0][0], u = red[0][1];
    for (int w = 1; w < kChunk / 32; w++) {
      add_hl(t, red[w][0]);
      u.x += red[w][1].x;
      u.y += red[w][1].y;
    }
    part_e[blockIdx.x] = t;
    part_q[blockIdx.x] = u;
  }
}

// one block per system: energy = 1/2 (sum of the system's item partials, in
// order); a system with a periodic axis and a net charge raises the
// non-neutral warning
__global__ void __launch_bounds__(1024) k_energy(const SysDev* __restrict__ sys, const float2* __restrict__ part_e,
                                                 const float2* __restrict__ part_q, double* __restrict__ energy,
                                                 int* __restrict__ status) {
  __shared__ float2 red[32][2];
  const SysDev& S = sys[blockIdx.x];
  float2 acc = make_float2(0.f, 0.f);
  float qs = 0.f, qa = 0.f;
  for (int i = threadIdx.x; i < S.nitem; i += blockDim.x) {
    add_hl(acc, part_e[S.item0 + i]);
    const float2 u = part_q[S.item0 + i];
    qs += u.x;
    qa += u.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    add_hl(acc, shfl_down_hl(acc, o));
    qs += __shfl_down_sync(0xffffffffu, qs, o);
    qa += __shfl_down_sync(0xffffffffu, qa, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = acc;
    red[threadIdx.x >> 5][1] = make_float2(qs, qa);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 t = red[0][0], u = red[0][1];
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
      add_hl(t, red[w][0]);
      u.x += red[w][1].x;
      u.y += red[w][1].y;
    }
    energy[blockIdx.x] = 0.5 * ((double)t.x + (double)t.y);
    if ((S.pbc[0] | S.pbc[1] | S.pbc[2]) && fabsf(u.x) > kNeutralTol * u.y) atomicOr(status, kDevNonNeutral);
  }
}

// Virial reduction, stage 1: block (s, b) of a (nsys x nslice) grid sums
// slice b of system s's partials (short-range per warp, then grid per tile)
// in a fixed order; stage 2: one block per system sums its slices and scales
// by g. Deterministic; the FP64 additions are spread over the whole GPU.

__device__ __forceinline__ void block_sum6(double (&acc)[6], double (*red)[6], double* out) {
  for (int c = 0; c < 6; c++) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) s += red[k][threadIdx.x];
    out[threadIdx.x] = s;
  }
}

__global__ void __launch_bounds__(256) k_virial_slices(const SysDev* __restrict__ sys,
                                                       const double* __restrict__ part_w0,
                                                       const double* __restrict__ part_wg,
                                                       const int* __restrict__ vitem_off, double* __restrict__ slices) {
  __shared__ double red[8][6];
  const int s = blockIdx.x, b = blockIdx.y, ns = gridDim.x, nslice = gridDim.y;
  const SysDev& S = sys[s];
  const int n0 = S.nitem * kChunkWarps;
  const int nb = vitem_off[s + 1] - vitem_off[s];
  const int nx = vitem_off[ns + 1 + s + 1] - vitem_off[ns + 1 + s];
  const int total = n0 + nb + nx;
  const int per = (total + nslice - 1) / nslice;
  const int lo = b * per, hi = min(total, lo + per);
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double* src;
    if (i < n0) src = part_w0 + 6 * ((long long)S.item0 * kChunkWarps + i);
    else if (i < n0 + nb) src = part_wg + 6 * (long long)(vitem_off[s] + (i - n0));
    else src = part_wg + 6 * (long long)(vitem_off[ns + 1 + s] + (i - n0 - nb));
    for (int c = 0; c < 6; c++) acc[c] += src[c];
  }
  block_sum6(acc, red, slices + 6 * ((long long)s * nslice + b));
}

__global__ void __launch_bounds__(64) k_virial_out(const double* __restrict__ slices, int nslice,
                                                   const double* __restrict__ grad, double* __restrict__ virial) {
  __shared__ double red[2][6];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const double* src = slices + 6 * (long long)blockIdx.x * nslice;
  for (int i = threadIdx.x; i < nslice; i += blockDim.x)
    for (int c = 0; c < 6; c++) acc[c] += src[6 * i + c];
  __shared__ double w[6];
  block_sum6(acc, red, w);
  __syncthreads();
  if (threadIdx.x == 0) {
    const double g = grad ? grad[blockIdx.x] : 1.0;
    double* V = virial + 9 * (long long)blockIdx.x;
    V[0] = g * w[0]; V[1] = g * w[3]; V[2] = g * w[4];
    V[3] = g * w[3]; V[4] = g * w[1]; V[5] = g * w[5];
    V[6] = g * w[4]; V[7] = g * w[5]; V[8] = g * w[2];
  }
}

// res (sorted) to the caller's order: phi_g, fsign F_g (fsign = -1 gives dE/dr =
// -F for dL/dE = 1, the same bits as k_backward_scale_res with dL/dE = 1).
// kGatherPer atoms of an item per thread, every index load issued before the
// first res load, so that each thread keeps kGatherPer dependent chains in
// flight.
constexpr int kGatherPer = 4, kGatherNT = kChunk / kGatherPer;

__global__ void __launch_bounds__(kGatherNT) k_outputs(const SysDev* __restrict__ sys, const AtomItem* __restrict__ items,
                                                       const int* __restrict__ iperm, const float4* __restrict__ res,
                                                       float* __restrict__ phi, float* __restrict__ forces,
                                                       float fsign) {
  AtomItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  int g[kGatherPer], k[kGatherPer];
#pragma unroll
  for (int r = 0; r < kGatherPer; r++) {
    const int slot = (int)threadIdx.x + r * kGatherNT, local = it.start + slot;
    g[r] = slot < it.count && local < S.n ? S.atom_off + local : -1;
    k[r] = g[r] >= 0 ? iperm[g[r]] : 0;
  }
  float4 v[kGatherPer];
#pragma unroll
  for (int r = 0; r < kGatherPer; r++) {
    if (g[r] >= 0 && !MSM_CHECK(S, k[r] >= S.atom_off && k[r] < S.atom_off + S.n)) g[r] = -1;
    v[r] = g[r] >= 0 ? res[k[r]] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int r = 0; r < kGatherPer; r++) {
    if (g[r] < 0) continue;
    if (phi) phi[g[r]] = v[r].x;
    if (forces) {
      forces[3 * (long long)g[r] + 0] = fsign * v[r].y;
      forces[3 * (long long)g[r] + 1] = fsign * v[r].z;
      forces[3 * (long long)g[r] + 2] = fsign * v[r].w;
    }
  }
}

// dE/dq = g phi, dE/dr = -g F from the forward's res, in the caller's order
// (kGatherPer atoms per thread, as k_outputs)
__global__ void __launch_bounds__(kGatherNT) k_backward_scale_res(const SysDev* __restrict__ sys,
                                                                  const AtomItem* __restrict__ items,
                                                                  const int* __restrict__ iperm,
                                                                  const float4* __restrict__ res,
                                                                  const double* __restrict__ grad,
                                                                  float* __restrict__ dE_dpos,
                                                                  float* __restrict__ dE_dq) {
  AtomItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  const float gr = (float)grad[it.sys];
  int g[kGatherPer], k[kGatherPer];
#pragma unroll
  for (int r = 0; r < kGatherPer; r++) {
    const int slot = (int)threadIdx.x + r * kGatherNT, local = it.start + slot;
    g[r] = slot < it.count && local < S.n ? S.atom_off + local : -1;
    k[r] = g[r] >= 0 ? iperm[g[r]] : 0;
  }
  float4 v[kGatherPer];
#pragma unroll
  for (int r = 0; r < kGatherPer; r++) {
    if (g[r] >= 0 && !MSM_CHECK(S, k[r] >= S.atom_off && k[r] < S.atom_off + S.n)) g[r] = -1;
    v[r] = g[r] >= 0 ? res[k[r]] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int r = 0; r < kGatherPer; r++) {
    if (g[r] < 0) continue;
    if (dE_dq) dE_dq[g[r]] = gr * v[r].x;
    if (dE_dpos) {
      dE_dpos[3 * (long long)g[r] + 0] = -gr * v[r].y;
      dE_dpos[3 * (long long)g[r] + 1] = -gr * v[r].z;
      dE_dpos[3 * (long long)g[r] + 2] = -gr * v[r].w;
    }
  }
}

// the same from the sorted potentials and fields (the backward recomputed the
// fields of a forward that skipped them)
__global__ void __launch_bounds__(kChunk) k_backward_scale(const SysDev* __restrict__ sys,
                                                           const AtomItem* __restrict__ items,
                                                           const int* __restrict__ perm,
                                                           const float4* __restrict__ xq,
                                                           const float* __restrict__ phi_sr,
                                                           const float* __restrict__ phi_lr,
                                                           const float4* __restrict__ f_sr,
                                                           const float4* __restrict__ f_lr,
                                                           const double* __restrict__ grad,
                                                           float* __restrict__ dE_dpos, float* __restrict__ dE_dq) {
  AtomItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  int local = it.start + threadIdx.x;
  if ((int)threadIdx.x >= it.count || local >= S.n) return;
  int k = S.atom_off + local;
  int g = perm[k];
  if (!MSM_CHECK(S, g >= S.atom_off && g < S.atom_off + S.n)) return;
  float gr = (float)grad[it.sys];
  if (dE_dq) dE_dq[g] = gr * (phi_sr[k] + phi_lr[k]);
  if (dE_dpos) {
    const float gq = -gr * xq[k].w;
    float4 a = f_sr[k], b = f_lr[k];
    dE_dpos[3 * (long long)g + 0] = gq * (a.x + b.x);
    dE_dpos[3 * (long long)g + 1] = gq * (a.y + b.y);
    dE_dpos[3 * (long long)g + 2] = gq * (a.z + b.z);
  }
}

// field_i = -grad phi(r_i) in the caller's atom order
__global__ void __launch_bounds__(kChunk) k_field(const SysDev* __restrict__ sys, const AtomItem* __restrict__ items,
                                                  const int* __restrict__ perm, const float4* __restrict__ f_sr,
                                                  const float4* __restrict__ f_lr, float* __restrict__ field) {
  AtomItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  int local = it.start + threadIdx.x;
  if ((int)threadIdx.x >= it.count || local >= S.n) return;
  int k = S.atom_off + local;
  int g = perm[k];
  float4 a = f_sr[k], b = f_lr[k];
  field[3 * (long long)g + 0] = a.x + b.x;
  field[3 * (long long)g + 1] = a.y + b.y;
  field[3 * (long long)g + 2] = a.z + b.z;
}

void launch_finalize(const Work& w, const Tables& t, const AtomItem* items, int nitems, bool forces, cudaStream_t s) {
  k_finalize<<<nitems, kChunk, 0, s>>>(t.sys, items, w.xq, w.phi_sr, w.phi_lr, w.f_sr, w.f_lr, forces, w.res,
                                       w.part_e, w.part_q);
}

void launch_outputs(const Work& w, const Tables& t, const AtomItem* items, int nitems, float* phi, float* forces,
                    float fsign, cudaStream_t s) {
  if (!phi && !forces) return;
  k_outputs<<<nitems, kGatherNT, 0, s>>>(t.sys, items, w.iperm, w.res, phi, forces, fsign);
}

void launch_energy(const Work& w, const Tables& t, int nsys, double* energy, cudaStream_t s) {
  k_energy<<<nsys, 1024, 0, s>>>(t.sys, w.part_e, w.part_q, energy, w.status);
}

// nslice (1 .. kVirialSlices) slices per system: about 1024 partials each for
// the largest system, so small batches do not launch idle blocks
void launch_virial_out(const Work& w, const Tables& t, int nsys, int nslice, const int* vitem_off,
                       const double* grad, double* virial, cudaStream_t s) {
  k_virial_slices<<<dim3(nsys, nslice), 256, 0, s>>>(t.sys, w.part_w0, w.part_wg, vitem_off, w.part_vs);
  k_virial_out<<<nsys, 64, 0, s>>>(w.part_vs, nslice, grad, virial);
}

void launch_backward_scale(const Work& w, const Tables& t, const AtomItem* items, int nitems,
                           const double* grad, float* dE_dpos, float* dE_dq, bool from_res, cudaStream_t s) {
  if (from_res)
    k_backward_scale_res<<<nitems, kGatherNT, 0, s>>>(t.sys, items, w.iperm, w.res, grad, dE_dpos, dE_dq);
  else
    k_backward_scale<<<nitems, kChunk, 0, s>>>(t.sys, items, w.perm, w.xq, w.phi_sr, w.phi_lr, w.f_sr, w.f_lr, grad,
                                               dE_dpos, dE_dq);
}

// upstream vectors of the forces into the sorted order, with the charge: us[k] = (u_perm[k], q_k)
__global__ void __launch_bounds__(kChunk) k_sort_u(const SysDev* __restrict__ sys, const AtomItem* __restrict__ items,
                                                   const int* __restrict__ perm, const float4* __restrict__ xq,
                                                   const float* __restrict__ u, float4* __restrict__ us) {
  AtomItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  int local = it.start + threadIdx.x;
  if ((int)threadIdx.x >= it.count || local >= S.n) return;
  int k = S.atom_off + local;
  long long g = perm[k];
  us[k] = make_float4(u[3 * g], u[3 * g + 1], u[3 * g + 2], xq[k].w);
}

// L = sum_k u_k . F_k:  dL/dq_i = u_i . E_i - psi_i,
//                        dL/dr_i = -q_i ((grad grad G) u_i + grad psi)_i,
// hg = ((H u)_grid, u . E), hs = ((H u)_short incl. grad psi_short, psi_short),
// phi_lr = psi_grid and f_lr = -grad psi_grid from the dipole grid chain.
__global__ void __launch_bounds__(kChunk) k_fvjp_final(const SysDev* __restrict__ sys,
                                                       const AtomItem* __restrict__ items,
                                                       const int* __restrict__ perm, const float4* __restrict__ xq,
                                                       const float4* __restrict__ hg, const float4* __restrict__ hs,
                                                       const float* __restrict__ psi_lr,
                                                       const float4* __restrict__ f_lr, float* __restrict__ dq,
                                                       float* __restrict__ dpos) {
  AtomItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  int local = it.start + threadIdx.x;
  if ((int)threadIdx.x >= it.count || local >= S.n) return;
  int k = S.atom_off + local;
  long long g = perm[k];
  const float4 a = hg[k], b = hs[k], c = f_lr[k];
  if (dq) dq[g] = a.w - b.w - psi_lr[k];
  if (dpos) {
    const float q = xq[k].w;
    dpos[3 * g + 0] = -q * (a.x + b.x - c.x);
    dpos[3 * g + 1] = -q * (a.y + b.y - c.y);
    dpos[3 * g + 2] = -q * (a.z + b.z - c.z);
  }
}

void launch_sort_u(const Work& w, const Tables& t, const AtomItem* items, int nitems, const float* u, float4* us,
                   cudaStream_t s) {
  k_sort_u<<<nitems, kChunk, 0, s>>>(t.sys, items, w.perm, w.xq, u, us);
}

void launch_fvjp_final(const Work& w, const Tables& t, const AtomItem* items, int nitems, const float4* hs, float* dq,
                       float* dpos, cudaStream_t s) {
  k_fvjp_final<<<nitems, kChunk, 0, s>>>(t.sys, items, w.perm, w.xq, w.f_sr, hs, w.phi_lr, w.f_lr, dq, dpos);
}

// potential VJP, before the evaluation with charges g: keep (E(q), q) per
// sorted atom in keep[k] and put g (caller's order -> sorted) in place of the
// charges in xq and uq
__global__ void __launch_bounds__(kChunk) k_pvjp_prep(const SysDev* __restrict__ sys,
                                                      const AtomItem* __restrict__ items, const int* __restrict__ perm,
                                                      const float* __restrict__ g, const float4* __restrict__ f_sr,
                                                      const float4* __restrict__ f_lr, float4* __restrict__ xq,
                                                      float4* __restrict__ uq, float4* __restrict__ keep) {
  AtomItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  int local = it.start + threadIdx.x;
  if ((int)threadIdx.x >= it.count || local >= S.n) return;
  int k = S.atom_off + local;
  const float4 a = f_sr[k], b = f_lr[k];
  const float gk = g[perm[k]];
  keep[k] = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, xq[k].w);
  xq[k].w = gk;
  uq[k].w = gk;
}

// potential VJP, after the evaluation with charges g: dL/dq = phi(g),
// dL/dr = -(g E(q) + q E(g)); the charges q go back into xq and uq
__global__ void __launch_bounds__(kChunk) k_pvjp_final(const SysDev* __restrict__ sys,
                                                       const AtomItem* __restrict__ items,
                                                       const int* __restrict__ perm, float4* __restrict__ xq,
                                                       float4* __restrict__ uq, const float4* __restrict__ keep,
                                                       const float* __restrict__ phi_sr,
                                                       const float* __restrict__ phi_lr,
                                                       const float4* __restrict__ f_sr,
                                                       const float4* __restrict__ f_lr, float* __restrict__ dq,
                                                       float* __restrict__ dpos) {
  AtomItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  int local = it.start + threadIdx.x;
  if ((int)threadIdx.x >= it.count || local >= S.n) return;
  int k = S.atom_off + local;
  long long gi = perm[k];
  const float4 eq = keep[k];
  const float gk = xq[k].w, qk = eq.w;
  if (dq) dq[gi] = phi_sr[k] + phi_lr[k];
  if (dpos) {
    const float4 a = f_sr[k], b = f_lr[k];
    dpos[3 * gi + 0] = -(gk * eq.x + qk * (a.x + b.x));
    dpos[3 * gi + 1] = -(gk * eq.y + qk * (a.y + b.y));
    dpos[3 * gi + 2] = -(gk * eq.z + qk * (a.z + b.z));
  }
  xq[k].w = qk;
  uq[k].w = qk;
}

void launch_pvjp_prep(const Work& w, const Tables& t, const AtomItem* items, int nitems, const float* g,
                      cudaStream_t s) {
  k_pvjp_prep<<<nitems, kChunk, 0, s>>>(t.sys, items, w.perm, g, w.f_sr, w.f_lr, w.xq, w.uq, w.vjp_u);
}

void launch_pvjp_final(const Work& w, const Tables& t, const AtomItem* items, int nitems, float* dq, float* dpos,
                       cudaStream_t s) {
  k_pvjp_final<<<nitems, kChunk, 0, s>>>(t.sys, items, w.perm, w.xq, w.uq, w.vjp_u, w.phi_sr, w.phi_lr, w.f_sr,
                                         w.f_lr, dq, dpos);
}

__global__ void k_fill_d(double* __restrict__ p, int n, double v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

void launch_fill(double* p, int n, double v, cudaStream_t s) {
  if (n > 0) k_fill_d<<<(n + 255) / 256, 256, 0, s>>>(p, n, v);
}

void launch_field(const Work& w, const Tables& t, const AtomItem* items, int nitems, float* field, cudaStream_t s) {
  k_field<<<nitems, kChunk, 0, s>>>(t.sys, items, w.perm, w.f_sr, w.f_lr, field);
}

}  // namespace msm
