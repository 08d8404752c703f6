// lq_xplan.cuh -- device side of the tiled <H> plans (XPlan): one CTA's
// evaluation of a plan's term groups on a 2^k-amplitude tile in shared
// memory, shared by the grid-wide tiled kernel (expval_tile_kernel) and the
// persistent batched launch (batch_kernel), which walks its own scratch
// state's tiles.  The terms, groups and their modes are those the host
// planner builds (Sec. V, the observable of Eq. expval).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "lq_device.cuh"
#include "lq_kernels.h"

namespace lq {

// Class-mode sums over this thread's indices j of the tile (j runs over the
// k - w bits outside x): amplitude i = expand(j) | dep[c] (lower x bits = class
// c, top x bit clear) pairs with i ^ x; sr[c] += Re conj(psi_i) psi_{i^x},
// si[c] += Im (as `part` asks), added to what sr and si hold.  Every class of
// an index is handled by the same thread, so the index expansion is shared.
template <int BLOCK, int W>
__device__ __forceinline__ void xp_class_sums(const double2* __restrict__ sm, uint32_t T,
                                              uint32_t x, int part, const uint32_t* dep,
                                              double* sr, double* si) {
  constexpr int NC = 1 << W;
  const uint32_t cnt = T >> (W + 1);
  // the x bit positions, ascending (zero bits are inserted lowest first)
  int pos[W + 1];
  {
    uint32_t mk = x;
#pragma unroll
    for (int b = 0; b <= W; b++) {
      pos[b] = __ffs(mk) - 1;
      mk &= mk - 1;
    }
  }
  constexpr int NL = NC < 2 ? NC : 2;   // classes loaded together (register budget)
  for (uint32_t j = threadIdx.x; j < cnt; j += BLOCK) {
    uint32_t a = j;
#pragma unroll
    for (int b = 0; b <= W; b++) a = insert0(a, pos[b]);
#pragma unroll
    for (int c0 = 0; c0 < NC; c0 += NL) {
      double2 A[NL], B[NL];
#pragma unroll
      for (int c = 0; c < NL; c++) {
        A[c] = sm[a | dep[c0 + c]];
        B[c] = sm[(a | dep[c0 + c]) ^ x];
      }
#pragma unroll
      for (int c = 0; c < NL; c++) {
        if (part != 2) sr[c0 + c] = fma(A[c].y, B[c].y, fma(A[c].x, B[c].x, sr[c0 + c]));
        if (part != 1) si[c0 + c] = fma(-A[c].y, B[c].x, fma(A[c].x, B[c].y, si[c0 + c]));
      }
    }
  }
}

// A run of class groups G[0..ng) of one width, part and coefficient block
// (the XX + YY groups of a uniform chain): their class sums add up before
// the coefficients are applied, so the fold costs 2^w FMAs per thread and
// tile for the whole run instead of for each group.
template <int BLOCK, int W>
__device__ __forceinline__ double xp_class_run(const double2* __restrict__ sm, uint32_t T,
                                               const XGroup* G, int ng,
                                               const double2* __restrict__ coef) {
  constexpr int NC = 1 << W;
  double sr[NC], si[NC];
#pragma unroll
  for (int c = 0; c < NC; c++) sr[c] = si[c] = 0.0;
  for (int r = 0; r < ng; r++) {
    uint32_t dep[NC];
    // deposit the class bits into the lower x bits (ascending)
#pragma unroll
    for (int c = 0; c < NC; c++) {
      uint32_t d = 0, mk = G[r].x & ~(1u << G[r].h);
      for (int b = 0; mk; b++) {
        const int bit = __ffs(mk) - 1;
        mk &= mk - 1;
        if (c >> b & 1) d |= 1u << bit;
      }
      dep[c] = d;
    }
    xp_class_sums<BLOCK, W>(sm, T, G[r].x, G[r].part, dep, sr, si);
  }
  const XGroup& G0 = G[0];
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < NC; c++) {
    const double2 C = coef[G0.coef + c];
    if (G0.part != 2) acc = fma(C.x, sr[c], acc);
    if (G0.part != 1) acc = fma(C.y, si[c], acc);
  }
  return acc;
}

// Per-CTA tables of the plan's diagonal group in `tab`: with coefficient
// classes, tab[off_c + p] = coefficient_c (count_c - 2 p) for p odd parities
// among the class's terms; with chunk tables, tab[c][v] = the sum over the
// chunk-c terms of c_t (-1)^popcount(v & z_t).  No barrier.
template <int BLOCK>
__device__ __forceinline__ void xp_tables(const XPlan& X, double* tab) {
  const uint32_t tid = threadIdx.x;
  if (X.diag < 0) return;
  if (X.dcls) {
    for (int c = 0, off = 0; c < X.dcls; off += X.dcount[c] + 1, c++)
      for (int p = tid; p <= X.dcount[c]; p += BLOCK)
        tab[off + p] = X.terms[X.dfirst[c]].c * (double)(X.dcount[c] - 2 * p);
  } else if (X.tables) {
    const int nch = (X.n + EXP_CHUNK_BITS - 1) / EXP_CHUNK_BITS;
    const XGroup& G = X.groups[X.diag];
    for (int e = tid; e < nch * 256; e += BLOCK) {
      const int c = e >> 8, v = e & 255;
      double s = 0.0;
      for (int t = G.first; t < G.first + G.count; t++) {
        if (X.terms[t].chunk != c + 1) continue;
        const uint32_t zc = (uint32_t)(X.terms[t].zg >> (EXP_CHUNK_BITS * c)) & 255u;
        s += (__popc((uint32_t)v & zc) & 1) ? -X.terms[t].c : X.terms[t].c;
      }
      tab[e] = s;
    }
  }
}

// Doubles of the tables xp_tables builds.
__host__ __device__ inline int xp_table_words(const XPlan& X) {
  if (X.diag < 0) return 0;
  if (X.dcls) {
    int w = 0;
    for (int c = 0; c < X.dcls; c++) w += X.dcount[c] + 1;
    return w;
  }
  return X.tables ? 256 * ((X.n + EXP_CHUNK_BITS - 1) / EXP_CHUNK_BITS) : 0;
}

// Global offsets (>> m) of pass Q's tile bits above its low run m:
// off(j) = hlo[j & 31] | hhi[j >> 5] (k - m <= XP_TILE_BITS - XP_LOW_BITS
// bits).  Threads 0-31 write them; the caller synchronises.
__device__ __forceinline__ void xp_offsets(const XPass& Q, uint32_t* hlo, uint32_t* hhi) {
  const uint32_t tid = threadIdx.x;
  const int m = Q.m, kh = Q.k - m;
  if (tid < 32) {
    const int kl = kh < 5 ? kh : 5;
    hlo[tid] = tid < (1u << kl) ? (uint32_t)(deposit(tid, Q.tbits + m, kl) >> m) : 0u;
    if (tid < (1u << (XP_TILE_BITS - XP_LOW_BITS - 5)))
      hhi[tid] = kh > 5 ? (uint32_t)(deposit((uint64_t)tid << 5, Q.tbits + m, kh) >> m) : 0u;
  }
}

// This thread's part of the plan's groups [Q.g0, Q.g1) on the tile sm
// (T = 2^Q.k amplitudes, CTA bits `base`; hlo/hhi from xp_offsets; coef:
// the plan's coefficient table, in shared or global memory; tab: the
// tables of xp_tables).  The caller synchronises before and after.
template <int BLOCK>
__device__ __forceinline__ double xp_tile(const double2* __restrict__ sm, uint32_t T,
                                          const XPlan& X, const XPass& Q, uint64_t base,
                                          const uint32_t* hlo, const uint32_t* hhi,
                                          const double2* __restrict__ coef,
                                          const double* __restrict__ tab) {
  const uint32_t tid = threadIdx.x;
  const int m = Q.m;
  const uint32_t lowmask = (1u << m) - 1u;
  const int nch = (X.n + EXP_CHUNK_BITS - 1) / EXP_CHUNK_BITS;
  auto hioff = [&](uint32_t j) { return hlo[j & 31u] | hhi[j >> 5]; };
  double acc = 0.0;
  for (int g = Q.g0; g < Q.g1; g++) {
    const XGroup& G = X.groups[g];
    if (G.mode == XG_CLASS) {
      int ng = 1;
      while (g + ng < Q.g1 && X.groups[g + ng].mode == XG_CLASS && X.groups[g + ng].w == G.w &&
             X.groups[g + ng].part == G.part && X.groups[g + ng].coef == G.coef)
        ng++;
      if (G.w == 1)
        acc += xp_class_run<BLOCK, 0>(sm, T, &G, ng, coef);
      else if (G.w == 2)
        acc += xp_class_run<BLOCK, 1>(sm, T, &G, ng, coef);
      else
        acc += xp_class_run<BLOCK, 2>(sm, T, &G, ng, coef);
      g += ng - 1;
    } else if (G.mode == XG_DIAG && X.dcls) {
      // per class: count the odd parities with integer operations, read the
      // class's sum from its table (K - 1 adds per amplitude)
      for (uint32_t s = tid; s < T; s += BLOCK) {
        const uint64_t gi = base | ((uint64_t)hioff(s >> m) << m) | (s & lowmask);
        const double2 v = sm[s];
        const double pr = fma(v.x, v.x, v.y * v.y);
        auto odd = [&](int c) {   // class-c terms with odd parity at gi
          int o = 0;
          for (int q = X.dfirst[c]; q < X.dfirst[c] + X.ddirect[c]; q++)
            o += __popcll(gi & X.terms[q].zg) & 1;
          for (int e = 0; e < X.dnd[c]; e++) {
            const int dl = X.ddel[c][e];
            o += __popcll((dl ? gi ^ (gi >> dl) : gi) & X.dmsk[c][e]);
          }
          return o;
        };
        double d = tab[odd(0)];
        for (int c = 1, off = X.dcount[0] + 1; c < X.dcls; off += X.dcount[c] + 1, c++)
          d += tab[off + odd(c)];
        acc = fma(d, pr, acc);
      }
    } else if (G.mode == XG_DIAG) {
      for (uint32_t s = tid; s < T; s += BLOCK) {
        const uint64_t gi = base | ((uint64_t)hioff(s >> m) << m) | (s & lowmask);
        const double2 v = sm[s];
        const double pr = fma(v.x, v.x, v.y * v.y);
        double d = 0.0;
        if (X.tables)
          for (int c = 0; c < nch; c++) d += tab[c * 256 + ((gi >> (EXP_CHUNK_BITS * c)) & 255)];
        for (int q = X.tables ? G.direct : G.first; q < G.first + G.count; q++) {
          const XTerm& Tm = X.terms[q];
          const uint32_t f = (uint32_t)(__popcll(gi & Tm.zg) & 1) << 31;
          d += xsign(Tm.c, f);
        }
        acc = fma(d, pr, acc);
      }
    } else {
      // table mode: index bit q = parity(j & z_q), CTA part per tile
      uint32_t gmask = 0, zl[XP_TABLE_TERMS];
#pragma unroll
      for (int q = 0; q < XP_TABLE_TERMS; q++) {
        zl[q] = q < G.count ? X.terms[G.first + q].zl : 0u;
        if (q < G.count) gmask |= (uint32_t)(__popcll(base & X.terms[G.first + q].zg) & 1) << q;
      }
      const uint32_t x = G.x;
      const int h = G.h;
      const double2* __restrict__ C = coef + G.coef;
      const int part = G.part;
      for (uint32_t j = tid; j < (T >> 1); j += BLOCK) {
        const uint32_t i0 = insert0(j, h), j0 = i0 ^ x;
        const double2 A = sm[i0], B = sm[j0];
        uint32_t idx = gmask;
#pragma unroll
        for (int q = 0; q < XP_TABLE_TERMS; q++) idx ^= (uint32_t)(__popc(j0 & zl[q]) & 1) << q;
        const double2 w = C[idx];
        if (part != 2) acc = fma(w.x, fma(A.x, B.x, A.y * B.y), acc);
        if (part != 1) acc = fma(w.y, fma(A.x, B.y, -(A.y * B.x)), acc);
      }
    }
  }
  return acc;
}

}  // namespace lq
