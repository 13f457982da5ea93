// Shared-memory Stockham FFT engine (radix 16 stages and at most one radix 2/4/8 stage, whose
// position the radix plan chooses).
//
// A "team" of L/16 threads transforms one row of length L (a power of two, 64..8192). Each
// thread keeps 16 complex values in registers; on entry and on exit thread t holds element
// t + q*(L/16) in v[q] (q = 0..15), natural order. The first stage reads the registers, every
// later stage reads the team's padded shared-memory row, and the last stage leaves its result
// in registers, so a caller can fuse zero-padding into the load, a spectral multiply between
// a forward and an inverse transform, and cropping into the store without extra passes.
//
// Stage s (sub-transform size Ns, radix R) of the autosort Stockham formulation: butterfly j
// reads x[j + r L/R] (r < R), multiplies element r by W_{Ns R}^{(j mod Ns) r}, takes an R-point
// DFT, and writes y[(j div Ns) Ns R + (j mod Ns) + r Ns]. Twiddles come from a table of
// exp(-2 pi i k r / (Ns R)) per stage, each rounded once from double precision on the host
// (conjugated for inverse transforms), laid out so that every warp's twiddle load is coalesced.
// Shared-memory rows carry one pad element per 16 so that the stride-16 writes of the first
// stage hit distinct banks.
//
// A row is private to its team, so the barriers inside a transform are team barriers (a warp
// barrier when the team fits in one warp, one named barrier per team otherwise): the teams of a
// block run independently between the block-wide barriers that callers place around the
// transposing loads and stores. Callers keep every thread on the FFT path (only global loads and
// stores are predicated), and a block holds at most 15 teams of 64 or more threads.
#pragma once

#include "xl_common.cuh"

namespace xl {

__host__ __device__ constexpr int cilog2(int n) { return n <= 1 ? 0 : 1 + cilog2(n >> 1); }
__host__ __device__ __forceinline__ constexpr int spad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int srow(int L) { return L + L / 16; }  // padded row length

// x * (DIR i): rotation by +-90 degrees (W_4 for the transform direction DIR = -1 / +1)
template <int DIR, typename C> __device__ __forceinline__ C rot90(C a) {
  return DIR < 0 ? mk(a.y, -a.x) : mk(-a.y, a.x);
}

template <int DIR, typename C> __device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a;
  a = cadd(a, b);
  b = csub(t, b);
}

// Pruned forms (HIN: the upper half of the inputs is zero and not read; HOUT: only the lower
// half of the outputs is formed, the upper half is left undefined). Exact: with zero inputs the
// full butterfly's additions of +0 would only turn a -0 into +0.
template <int DIR, bool HIN = false, bool HOUT = false, typename C>
__device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  if constexpr (HIN) {
    const C d13 = rot90<DIR>(a1);
    const C x0 = a0, x1 = a1;
    a0 = cadd(x0, x1);
    a1 = cadd(x0, d13);
    if constexpr (!HOUT) {
      a2 = csub(x0, x1);
      a3 = csub(x0, d13);
    }
  } else {
    C s02 = cadd(a0, a2), d02 = csub(a0, a2);
    C s13 = cadd(a1, a3), d13 = rot90<DIR>(csub(a1, a3));
    a0 = cadd(s02, s13);
    a1 = cadd(d02, d13);
    if constexpr (!HOUT) {
      a2 = csub(s02, s13);
      a3 = csub(d02, d13);
    }
  }
}

// x * exp(DIR i pi/4)
template <int DIR, typename C> __device__ __forceinline__ C w8_1(C a) {
  typedef decltype(a.x) T;
  const T h = (T)0.70710678118654752440084436210484903;
  return DIR < 0 ? mk((a.x + a.y) * h, (a.y - a.x) * h) : mk((a.x - a.y) * h, (a.y + a.x) * h);
}
// x * exp(DIR i 3pi/4)
template <int DIR, typename C> __device__ __forceinline__ C w8_3(C a) {
  typedef decltype(a.x) T;
  const T h = (T)0.70710678118654752440084436210484903;
  return DIR < 0 ? mk((-a.x + a.y) * h, (-a.y - a.x) * h) : mk((-a.x - a.y) * h, (-a.y + a.x) * h);
}

// In-place 8-point DFT of v[o + s*k], k = 0..7 (natural order in and out); HIN / HOUT as dft4.
template <int DIR, int S, bool HIN = false, bool HOUT = false, typename C>
__device__ __forceinline__ void dft8s(C* v) {
  C e0 = v[0], e1 = v[2 * S], e2, e3;
  C o0 = v[S], o1 = v[3 * S], o2, o3;
  if constexpr (!HIN) {
    e2 = v[4 * S];
    e3 = v[6 * S];
    o2 = v[5 * S];
    o3 = v[7 * S];
  }
  dft4<DIR, HIN>(e0, e1, e2, e3);
  dft4<DIR, HIN>(o0, o1, o2, o3);
  o1 = w8_1<DIR>(o1);
  o2 = rot90<DIR>(o2);
  o3 = w8_3<DIR>(o3);
  v[0] = cadd(e0, o0);
  v[S] = cadd(e1, o1);
  v[2 * S] = cadd(e2, o2);
  v[3 * S] = cadd(e3, o3);
  if constexpr (!HOUT) {
    v[4 * S] = csub(e0, o0);
    v[5 * S] = csub(e1, o1);
    v[6 * S] = csub(e2, o2);
    v[7 * S] = csub(e3, o3);
  }
}

// In-place 16-point DFT of v[s*k], k = 0..15: two 8-point DFTs of the even and odd samples
// and the W_16^k combination; HIN / HOUT as dft4.
template <int DIR, int S, bool HIN = false, bool HOUT = false, typename C>
__device__ __forceinline__ void dft16s(C* v) {
  typedef decltype(v[0].x) T;
  C e[8], o[8];
#pragma unroll
  for (int k = 0; k < (HIN ? 4 : 8); ++k) {
    e[k] = v[2 * k * S];
    o[k] = v[(2 * k + 1) * S];
  }
  dft8s<DIR, 1, HIN>(e);
  dft8s<DIR, 1, HIN>(o);
  const T c1 = (T)0.92387953251128675612818318939678829;  // cos(pi/8)
  const T s1 = (T)0.38268343236508977172845998403039887;  // sin(pi/8)
  const T sd = (T)DIR;
  // W16^k = cos(pi k / 8) + DIR i sin(pi k / 8)
  o[1] = cmul(o[1], mk(c1, sd * s1));
  o[2] = w8_1<DIR>(o[2]);
  o[3] = cmul(o[3], mk(s1, sd * c1));
  o[4] = rot90<DIR>(o[4]);
  o[5] = cmul(o[5], mk(-s1, sd * c1));
  o[6] = w8_3<DIR>(o[6]);
  o[7] = cmul(o[7], mk(-c1, sd * s1));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k * S] = cadd(e[k], o[k]);
    if constexpr (!HOUT) v[(k + 8) * S] = csub(e[k], o[k]);
  }
}

template <int R, int DIR, int S, bool HIN = false, bool HOUT = false, typename C>
__device__ __forceinline__ void dftR(C* v) {
  if constexpr (R == 16) dft16s<DIR, S, HIN, HOUT>(v);
  else if constexpr (R == 8) dft8s<DIR, S, HIN, HOUT>(v);
  else if constexpr (R == 4) dft4<DIR, HIN, HOUT>(v[0], v[S], v[2 * S], v[3 * S]);
  else if constexpr (HIN) v[S] = v[0];  // R == 2 with a zero second input
  else if constexpr (HOUT) v[0] = cadd(v[0], v[S]);
  else dft2<DIR>(v[0], v[S]);
}

// Pruning of a whole transform (template argument PRUNE of team_fft): PRUNE_IN, the inputs
// q >= 8 (the upper half of the row) are zero and not read; PRUNE_OUT, only the outputs q < 8
// (the lower half) are formed, v[8..15] are left undefined. The zero-padded transforms of the RS
// convolution take both: half of every input row is padding and half of every output is cropped.
constexpr int PRUNE_IN = 1, PRUNE_OUT = 2;

// Radix plan of a length-L transform: L = 16^a 2^REM (REM = log2 L mod 4). Every stage has radix
// 16 except one of radix 2^REM (when REM > 0), which sits last (PLAN 0), first (PLAN 1) or second
// (PLAN 2; the same as PLAN 0 for two-stage lengths). Each thread keeps 16 values, so a stage of
// radix R runs 16 / R butterflies a thread; all plans take the same number of stages, shared-
// memory exchanges and flops and differ in their twiddle and bank patterns (the autotuner picks).
template <int L, int PLAN = 0> struct FFTShape {
  static constexpr int LOG = cilog2(L);
  static constexpr int N16 = LOG / 4;              // radix-16 stages
  static constexpr int REM = LOG % 4;              // log2 of the odd stage's radix (0: none)
  static constexpr int NST = N16 + (REM ? 1 : 0);  // number of stages
  static constexpr int TT = L / 16;                // threads per team
  static constexpr int POS = REM == 0 ? -1 : (PLAN == 1 ? 0 : (PLAN == 2 && NST > 2 ? 1 : NST - 1));
  static constexpr int radix(int s) { return s == POS ? (1 << REM) : 16; }
  static constexpr int ns(int s) {  // sub-transform size before stage s
    int n = 1;
    for (int i = 0; i < s; ++i) n *= radix(i);
    return n;
  }
  static_assert((1 << LOG) == L && L >= 64 && L <= 8192, "FFT length: power of two in [64, 8192]");
  static_assert(PLAN >= 0 && PLAN <= 2, "radix plan: 0, 1 or 2");
};

// Twiddle table layout: for every stage S >= 1 (sub-transform size Ns, radix R) a block of
// R x Ns entries tw[off_S + r Ns + k] = exp(-2 pi i k r / (Ns R)), each rounded once from double
// precision on the host. For a fixed r the lanes of a warp (consecutive butterflies, consecutive
// k) read consecutive entries, so every twiddle load is coalesced.
template <int L, int PLAN = 0> __host__ __device__ constexpr int tw_stage_offset(int S) {
  typedef FFTShape<L, PLAN> Sh;
  int off = 0;
  for (int s = 1; s < S; ++s) off += Sh::radix(s) * Sh::ns(s);
  return off;
}

// Multiplies v[B r] by W_{Ns R}^{k r}, r = 1..R-1 (conjugated for inverse transforms);
// `col` points at entry (r = 0, k) of the stage block.
template <int R, int B, int Ns, typename C>
__device__ __forceinline__ void apply_twiddles(C* v, const C* __restrict__ col, bool inv) {
#pragma unroll
  for (int r = 1; r < R; ++r) {
    C w = __ldg(col + r * Ns);
    if (inv) w = cconj(w);
    v[r * B] = cmul(v[r * B], w);
  }
}

// Barrier of the team that owns a row (ids 1.. of the named barriers; 0 is __syncthreads).
template <int L> __device__ __forceinline__ void team_sync() {
  constexpr int TT = L / 16;
  if constexpr (TT <= 32) {
    __syncwarp();
  } else {
    const int id = 1 + (int)(threadIdx.x / TT);
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(TT) : "memory");
  }
}
// Whether a block of `threads` threads fits the team barriers of length-L transforms.
template <int L> __host__ __device__ constexpr bool team_barriers_fit(int threads) {
  return L / 16 <= 32 || threads / (L / 16) <= 15;
}

// Stage S (>= 1) of the transform under radix plan PLAN.
template <int L, int DIR, int S, int PLAN, int PRUNE, typename C>
__device__ __forceinline__ void fft_stage(C (&v)[16], C* sm, int t, const C* __restrict__ tw) {
  typedef FFTShape<L, PLAN> Sh;
  constexpr bool last = (S == Sh::NST - 1);
  constexpr int R = Sh::radix(S);
  constexpr int B = 16 / R;
  constexpr int Ns = Sh::ns(S);
  constexpr int TT = Sh::TT;
  team_sync<L>();
#pragma unroll
  for (int b = 0; b < B; ++b)
#pragma unroll
    for (int r = 0; r < R; ++r) v[b + B * r] = sm[spad(t + (b + B * r) * TT)];
  if constexpr (!last) team_sync<L>();
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = t + b * TT;
    const int k = j & (Ns - 1);
    apply_twiddles<R, B, Ns>(v + b, tw + tw_stage_offset<L, PLAN>(S) + k, DIR > 0);
    dftR<R, DIR, B, false, last && (PRUNE & PRUNE_OUT) != 0>(v + b);
  }
  if constexpr (!last) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = t + b * TT;
      const int base = (j / Ns) * Ns * R + (j & (Ns - 1));
#pragma unroll
      for (int r = 0; r < R; ++r) sm[spad(base + r * Ns)] = v[b + B * r];
    }
    fft_stage<L, DIR, (S + 1 < Sh::NST ? S + 1 : S), PLAN, PRUNE>(v, sm, t, tw);
  }
}

// Row pitch (in elements) of a block's shared-memory rows: at least srow(L), with the residue
// modulo 16 that puts the rows one warp phase touches in the transposed stores and loads in
// distinct banks. Those loops give each group of G = min(32 / element bytes, ROWS) lanes one
// 32-byte sector (G consecutive rows of one column): G = 4 (complex64) and G = 2 (complex128)
// want rows 4 elements apart modulo 16, G = 2 for complex64 wants 8.
__host__ __device__ constexpr int tpitch(int L, int CS, int ROWS) {
  return srow(L) + ((((CS == 8 && (32 / CS < ROWS ? 32 / CS : ROWS) == 2) ? 8 : 4) - srow(L) % 16) + 16) % 16;
}

// Transposed block store by a block of ROWS teams of length-L transforms (ROWS * L / 16 threads):
// rows 0..ROWS-1 of the block's shared memory (pitch P) hold the first n_out entries of ROWS
// transforms; element j of row r goes to dst[j * ld + c0 + r] (r with c0 + r < n_cols). Lanes
// are grouped so that each warp instruction writes whole 32-byte sectors (G = 32 / sizeof(C)
// consecutive rows of one j per group of lanes). A thread keeps one row r and steps j by
// JS = threads / G, so its row test, addresses and padding are computed once and advanced by
// fixed steps; with n_out known at compile time the loop unrolls completely.
template <int L, int ROWS, int P, typename C>
__device__ __forceinline__ void store_rows_transposed(const C* sm, int n_out, C* __restrict__ dst,
                                                      int64_t ld, int c0, int n_cols) {
  constexpr int NT = ROWS * (L / 16);
  constexpr int G0 = 32 / (int)sizeof(C);
  constexpr int G = G0 < ROWS ? G0 : ROWS;
  constexpr int LG = G == 4 ? 2 : (G == 2 ? 1 : 0);
  constexpr int JS = NT / G;
  static_assert(NT % G == 0, "transposed store: thread count and sector groups");
  const int rr = threadIdx.x & (G - 1), j0 = threadIdx.x >> LG;
  auto soff = [&](int k) {  // padded offset of j0 + k JS from j0
    if constexpr (JS % 16 == 0) return k * (JS + JS / 16);
    else return spad(j0 + k * JS) - spad(j0);
  };
  const int nfull = n_out / JS;  // iterations in which every thread's j is below n_out
  const int64_t dstep = (int64_t)JS * ld;
#pragma unroll 1
  for (int grp = 0; grp < ROWS / G; ++grp) {
    const int r = grp * G + rr;
    if (c0 + r < n_cols) {
      const C* s = sm + r * P + spad(j0);
      C* d = dst + (int64_t)j0 * ld + c0 + r;
#pragma unroll 4
      for (int k = 0; k < nfull; ++k) d[k * dstep] = s[soff(k)];
      if (j0 + nfull * JS < n_out) d[nfull * dstep] = s[soff(nfull)];
    }
  }
}

// Transposed block load (inverse of the store, same block shape): row r of shared memory gets
// src[j * ld + c0 + r] for j < n_in and zero for n_in <= j < n_fill. Callers synchronise the
// block before reading the rows. ASYNC: asynchronous global-to-shared copies (zero-filled where
// there is no source element), so that a thread issues all of its copies before it waits once
// (measured faster for RS pass 3, slower for the CZT adjoint passes, which keep plain loads).
template <int L, int ROWS, int P, typename C, bool ASYNC = false>
__device__ __forceinline__ void load_rows_transposed(C* sm, int n_in, int n_fill,
                                                     const C* __restrict__ src, int64_t ld, int c0,
                                                     int n_cols) {
  typedef decltype(sm[0].x) T;
  constexpr int NT = ROWS * (L / 16);
  constexpr int G0 = 32 / (int)sizeof(C);
  constexpr int G = G0 < ROWS ? G0 : ROWS;
  constexpr int LG = G == 4 ? 2 : (G == 2 ? 1 : 0);
  constexpr int JS = NT / G;
  static_assert(NT % G == 0, "transposed load: thread count and sector groups");
  const int rr = threadIdx.x & (G - 1), j0 = threadIdx.x >> LG;
  auto soff = [&](int k) {
    if constexpr (JS % 16 == 0) return k * (JS + JS / 16);
    else return spad(j0 + k * JS) - spad(j0);
  };
  const int nfull = n_fill / JS;
  const int64_t sstep = (int64_t)JS * ld;
  auto one = [&](C* s, const C* g, bool ok) {
    if constexpr (ASYNC) {
      const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
      asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sa),
                   "l"(ok ? g : src),  // a valid address when nothing is read
                   "n"((int)sizeof(C)), "r"(ok ? (int)sizeof(C) : 0)
                   : "memory");
    } else {
      *s = ok ? *g : mk((T)0, (T)0);
    }
  };
#pragma unroll 1
  for (int grp = 0; grp < ROWS / G; ++grp) {
    const int r = grp * G + rr;
    const bool col = c0 + r < n_cols;
    C* s = sm + r * P + spad(j0);
    const C* g = src + (int64_t)j0 * ld + c0 + r;
#pragma unroll 4
    for (int k = 0; k < nfull; ++k)
      one(s + soff(k), g + k * sstep, col && j0 + k * JS < n_in);
    if (j0 + nfull * JS < n_fill)
      one(s + soff(nfull), g + nfull * sstep, col && j0 + nfull * JS < n_in);
  }
  if constexpr (ASYNC) {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  }
}

// Asks L2 to fetch the bytes [p, p + bytes) ahead of their loads (one bulk prefetch: no
// registers held, no completion to wait for). The range is shrunk to whole 16-byte units inside
// it, as the instruction requires; the ends are read by the loads themselves.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
  const uintptr_t s = ((uintptr_t)p + 15) & ~(uintptr_t)15;
  const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
  if (e > s)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(s), "r"((unsigned)(e - s))
                 : "memory");
}

// Shared-memory address of a generic pointer (for bulk copies and barriers).
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
// Iteration bound of the waits on bulk-copy barriers (a wait that runs out reports an error).
constexpr unsigned kWaitLimit = 1u << 26;

// Thread-private 16-element stash (element q of thread t is row element t + q L/16), in a shared
// memory row or in registers.
template <typename C, int TT, bool SMEM> struct Stash {
  C r[16];
  __device__ __forceinline__ void init(C*, int) {}
  __device__ __forceinline__ C get(int q) const { return r[q]; }
  __device__ __forceinline__ void set(int q, C v) { r[q] = v; }
};
template <typename C, int TT> struct Stash<C, TT, true> {
  C* p;
  int t;
  __device__ __forceinline__ void init(C* row, int tt) { p = row; t = tt; }
  __device__ __forceinline__ C get(int q) const { return p[spad(t + q * TT)]; }
  __device__ __forceinline__ void set(int q, C v) { p[spad(t + q * TT)] = v; }
};

// Full length-L transform of one row held by a team (see the file comment for the layout).
// sm: the team's padded shared-memory row (srow(L) elements); tw: the twiddle table of plan PLAN.
// The team barrier after the register-only first stage orders its shared-memory writes after
// every read of the row by a previous transform (a forward transform's last stage reads the row just
// before a caller multiplies and runs the inverse transform on the same row).
template <int L, int DIR, int PLAN = 0, int PRUNE = 0, typename C>
__device__ __forceinline__ void team_fft(C (&v)[16], C* sm, int t, const C* __restrict__ tw) {
  typedef FFTShape<L, PLAN> Sh;
  constexpr int R0 = Sh::radix(0), B0 = 16 / R0, TT = Sh::TT;
  // stage 0 (Ns = 1, no twiddles) on the registers: butterfly j = t + b TT writes y[j R0 + r];
  // with PRUNE_IN its inputs r >= R0 / 2 (q = b + B0 r >= 8) are the zero padding
#pragma unroll
  for (int b = 0; b < B0; ++b) dftR<R0, DIR, B0, (PRUNE & PRUNE_IN) != 0>(v + b);
  team_sync<L>();
#pragma unroll
  for (int b = 0; b < B0; ++b)
#pragma unroll
    for (int r = 0; r < R0; ++r) sm[spad((t + b * TT) * R0 + r)] = v[b + B0 * r];
  fft_stage<L, DIR, 1, PLAN, PRUNE>(v, sm, t, tw);
}

}  // namespace xl
