// Mixed-precision right-hand side with the D and LIFT contraction on the fifth-generation
// tensor cores (tcgen05): operands in shared memory in the UMMA K-major layout, the
// accumulator in tensor memory (TMEM), MMAs issued by one thread and completed through an
// mbarrier, and the FP64 RK update from a shared-memory copy of the accumulator.
//
// Tile: 25 elements, rows r = 5 e + v (125 of the MMA's M = 128 rows; rows 125..127 are never
// read), columns = output nodes i (N = NPAD = Np rounded up to 16).  The reduction runs over
// chunks: three volume chunks of KV = NPAD columns (reference directions r, s, t: the
// contravariant fluxes against -D_r, -D_s, -D_t) and one or two surface chunks of KS columns
// (Fscale g against LIFT; one chunk of 48 at N = 3).  Each chunk is produced by all threads
// into one shared-memory slot, then contracted by width/16 k-steps of the six split-BF16
// products while nothing else may touch the slot; the blocks resident on an SM (two at N = 3)
// overlap one block's production with another's MMAs.  A tile's own node records are staged in
// shared memory one tile ahead (TMA bulk copies issued under the previous tile's last MMA
// round), where that costs no resident block.  Operand columns past Np (volume) or past the
// face-node count (last surface chunk) hold zeros or stale finite values from an earlier chunk;
// the operator table is zero there, so they contribute nothing.
#pragma once

#include "dg_mixed.cuh"
#include "dg_umma.cuh"

namespace dg {
namespace tc {

using mixk::MixedCase;
using kern::GS;

// Tiles of the Navier-Stokes right-hand side, with or without artificial viscosity: they read the
// BR1 viscous-flux records.
__host__ __device__ constexpr bool tile_ns(int PHYS) {
  return PHYS == kern::NAVIER_STOKES || PHYS == kern::NS_AV;
}

// One thread's L2 prefetch of a tile's contiguous inputs (the node records or, for a mixture,
// the float state copy, pressure and sound speed; the viscous-flux records for Navier-Stokes),
// geometry and neighbour map of elements [e0, e0 + nel).
__device__ __forceinline__ void prefetch_tile_inputs(const MixedCase& c, int e0, int nel, int Np, int NF, bool mix,
                                                     bool ns) {
  const size_t KNp = (size_t)c.K * Np, base = (size_t)e0 * Np, nn = (size_t)nel * Np;
  if (mix) {
    prefetch_l2(c.mrec + 4 * base, nn * 64);
  } else {
    prefetch_l2(c.node + 2 * base, nn * 32);
    if (ns) {
      prefetch_l2(c.fv4 + 2 * base, nn * 32);
      prefetch_l2(c.fvz + base, nn * 4);
    }
  }
  prefetch_l2(c.geo + (size_t)e0 * GS, (size_t)nel * GS * 4);
  prefetch_l2(c.vmapP + (size_t)e0 * NF, (size_t)nel * NF * 4);
}

// ---- tile configuration --------------------------------------------------------------------
constexpr int round16(int x) { return (x + 15) / 16 * 16; }

// Single-case threads per tile (the batched form's autotuner picks among two compiled
// candidates per order; these are its choices on the benchmark workloads).
__host__ __device__ constexpr int default_nt(int N) { return N == 1 ? 128 : (N == 4 ? 448 : 256); }
__host__ __device__ constexpr int default_vis_nt(int N) { return N == 1 ? 128 : (N == 2 ? 128 : (N == 3 ? 512 : 896)); }

// Blocks per SM that the compiler's register budget aims at: the shared-memory limit, the
// thread limit, and no fewer than min_regs registers per thread.
__host__ __device__ constexpr int aim_blocks(int smem, int nt, int min_regs = 64) {
  const int by_smem = (228 * 1024) / (smem + 1024), by_thr = 2048 / nt, by_reg = 65536 / (nt * min_regs);
  const int m = by_smem < by_thr ? by_smem : by_thr;
  const int r = m < by_reg ? m : by_reg;
  return r < 1 ? 1 : r;
}

// Whether a tile layout ending at `end_vm` bytes (with the staged neighbour map) keeps as many
// resident blocks per SM as the one ending at `end` (without it).
__host__ __device__ constexpr bool vm_fits(int end, int end_vm, int nt, int min_regs) {
  return aim_blocks(end_vm + 24, nt, min_regs) >= aim_blocks(end + 24, nt, min_regs);
}

// Columns of a surface chunk.  At N = 3 the 40 face nodes of an element go into one chunk of
// 48 columns instead of chunks of 32 and 8: one MMA round trip and one gather pass less per
// tile, for a wider operand slot that still leaves the resident blocks per SM unchanged.  In the
// right-hand-side tile (merge_n2) the same holds at N = 2, 24 face nodes in one chunk of 32
// instead of 16 and 8.  N = 4 keeps the volume width: the wider slot would cost half the
// resident blocks.  A function of the order (and tile kind) alone, so that every tile variant
// of an order shares one operator table.
__host__ __device__ constexpr int surface_cols(int N, int KV, int NF, bool merge_n2 = false) {
  return (N == 3 || (merge_n2 && N == 2)) ? round16(NF) : KV;
}

// Threads per tile of a mixture (13 rows per element, 9 elements per tile): about one node per thread.
__host__ __device__ constexpr int mixture_nt(int N) { return N <= 2 ? 128 : (N == 3 ? 192 : 320); }

template <int N, int NT_ = default_nt(N), int V_ = 5>
struct Cfg {
  using O = kern::Ord<N>;
  static constexpr int ORDER = N, V = V_;
  static constexpr int Np = O::Np, Nfp = O::Nfp, NF = O::NF;
  static constexpr int E = 128 / V, ROWS = 128;  // rows (element, variable) of one MMA tile
  static constexpr int KV = round16(Np), NPAD = KV;
  // surface columns per chunk (surface_cols: all face nodes in one chunk at N = 3)
  static constexpr int NVOL = 3, KS = surface_cols(N, KV, NF, true), KA = KS > KV ? KS : KV;
  static constexpr int NSURF = (NF + KS - 1) / KS, NCHUNK = NVOL + NSURF, KB = NVOL * KV + NSURF * KS;
  // operand slot: 3 terms x 128 rows x KA columns; core matrices adjacent in K are 144 B apart
  // (not 128) so that the 16 B rows written by consecutive node threads fall in distinct banks
  static constexpr int A_LBO = 144, A_SBO = (KA / 8) * A_LBO, A_TERM = 16 * A_SBO;
  // operator table: 3 terms x NPAD rows x KB columns
  static constexpr int B_LBO = 128, B_SBO = (KB / 8) * B_LBO, B_TERM = (NPAD / 8) * B_SBO;
  static constexpr int CS = NPAD + 1;  // row stride (floats) of the accumulator copy
  static constexpr int TMEM_COLS = NPAD <= 32 ? 32 : 64;
  static constexpr int NT = NT_;
  static constexpr int NODES = E * Np, NPT = (NODES + NT - 1) / NT;
  static constexpr uint32_t IDESC = idesc_bf16(ROWS, NPAD);
  // shared-memory layout (bytes)
  static constexpr int OFF_B = 0, OFF_A = 3 * B_TERM, OFF_GEO = OFF_A + 3 * A_TERM;
  static constexpr int OFF_FM = OFF_GEO + E * GS * 4;
  // registers a thread gets at least: a node's three 5-variable fluxes stay live over three MMA
  // rounds (about 110 registers without spilling, which would go to L2: the L1 left beside this
  // much shared memory is small); a mixture node holds 3 x 13 fluxes (128: four blocks of 128
  // threads per SM at N = 2, measured faster than five spilling ones and three of 160 registers).
  // Perfect gas at N = 4 (448 threads): one block per SM at 128 registers with staged records,
  // measured faster (0.81 against 0.91 ms on 196,608 tets) than two spilling blocks of 72.
  static constexpr int MIN_REGS = V > 5 ? (NT <= 192 ? 128 : 96) : (NT <= 256 ? 96 : (NT <= 448 ? 128 : 64));
  // the tile's neighbour map, staged in shared memory where that costs no resident block
  static constexpr int OFF_VM = (OFF_FM + NF * 4 + 15) / 16 * 16, VM_BYTES = E * NF * 4;
  static constexpr bool VM = vm_fits(OFF_FM + NF * 4, OFF_VM + VM_BYTES, NT, MIN_REGS);
  static constexpr int END_VM = VM ? OFF_VM + VM_BYTES : OFF_FM + NF * 4;
  // perfect gas: the tile's own node records, viscous-flux records and Q_z values, staged one
  // tile ahead (where that costs no resident block): [E Np] x 2 float4, [E Np] x 2 float4, [E Np]
  static constexpr int OFF_ST = (END_VM + 15) / 16 * 16, ST_BYTES = E * Np * 64 + (E * Np * 4 + 15) / 16 * 16;
  static constexpr bool STAGE = V == 5 && VM && vm_fits(END_VM, OFF_ST + ST_BYTES, NT, MIN_REGS);
  static constexpr int OFF_BAR = ((STAGE ? OFF_ST + ST_BYTES : END_VM) + 7) / 8 * 8;
  static constexpr int SMEM = OFF_BAR + 24;
  static constexpr int MINB = aim_blocks(SMEM, NT, MIN_REGS);
  static_assert(ROWS * CS * 4 <= 3 * A_TERM, "the accumulator copy must fit in the operand slot");
  static_assert(ROWS * CS % 4 == 0, "the accumulator copy is cleared in 16 B words");
  static_assert(NPAD <= TMEM_COLS, "TMEM columns");
  static_assert(OFF_A % 16 == 0 && A_TERM % 16 == 0 && B_TERM % 16 == 0, "UMMA operands need 16 B alignment");
  static_assert(NT % 32 == 0 && NT >= 128 && NT <= 1024, "whole warps, at least the four TMEM lane quarters");
};

// Byte offset of (row, k) in a K-major no-swizzle operand.
__device__ __forceinline__ int umma_off(int row, int k, int lbo, int sbo) {
  return (row >> 3) * sbo + (k >> 3) * lbo + (row & 7) * 16 + (k & 7) * 2;
}

// Split FP32 value v into three BF16 terms (v = hi + mid + lo to 24 bits) stored at `off` of
// the three term arrays (term stride ts bytes).
__device__ __forceinline__ void put3_umma(unsigned char* A, int ts, int off, float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(h);
  const __nv_bfloat16 m = __float2bfloat16_rn(r1);
  const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
  *reinterpret_cast<__nv_bfloat16*>(A + off) = h;
  *reinterpret_cast<__nv_bfloat16*>(A + ts + off) = m;
  *reinterpret_cast<__nv_bfloat16*>(A + 2 * ts + off) = l;
}

template <class C_>
struct Smem {
  unsigned char* B;
  unsigned char* A;
  float* C;  // accumulator copy, aliases the operand slot once the tile's MMAs are done
  float* geo;
  int* fm;
  int* vm;  // the tile's neighbour map [E][NF] (only when C_::VM)
  // staged node records of the tile (only when C_::STAGE)
  float4* st_node;
  float4* st_fv4;
  float* st_fvz;
  float2* st_temp;  // BR1 tile: the staged temperature pairs (after the node records)
  uint64_t* bar;     // MMA completion
  uint64_t* st_bar;  // staging copies
  uint32_t* tmem;
  int* abort;
  __device__ explicit Smem(unsigned char* raw) {
    B = raw + C_::OFF_B;
    A = raw + C_::OFF_A;
    C = reinterpret_cast<float*>(A);
    geo = reinterpret_cast<float*>(raw + C_::OFF_GEO);
    fm = reinterpret_cast<int*>(raw + C_::OFF_FM);
    vm = reinterpret_cast<int*>(raw + C_::OFF_VM);
    st_node = reinterpret_cast<float4*>(raw + C_::OFF_ST);
    st_fv4 = st_node + 2 * C_::E * C_::Np;
    st_fvz = reinterpret_cast<float*>(st_fv4 + 2 * C_::E * C_::Np);
    st_temp = reinterpret_cast<float2*>(st_fv4);
    bar = reinterpret_cast<uint64_t*>(raw + C_::OFF_BAR);
    tmem = reinterpret_cast<uint32_t*>(raw + C_::OFF_BAR + 8);
    abort = reinterpret_cast<int*>(raw + C_::OFF_BAR + 12);
    st_bar = reinterpret_cast<uint64_t*>(raw + C_::OFF_BAR + 16);
  }
};

// Block set-up: operator table, face map, a zeroed operand slot (no NaN patterns in columns
// that no chunk writes), the mbarrier and the TMEM accumulator.
template <class C_>
__device__ __forceinline__ void block_setup(const Smem<C_>& S, const uint4* __restrict__ b_g,
                                            const int32_t* __restrict__ fmask_g) {
  const int tid = threadIdx.x;
  uint4* Bs = reinterpret_cast<uint4*>(S.B);
  for (int i = tid; i < 3 * C_::B_TERM / 16; i += blockDim.x) Bs[i] = b_g[i];
  uint4* As = reinterpret_cast<uint4*>(S.A);
  for (int i = tid; i < 3 * C_::A_TERM / 16; i += blockDim.x) As[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < C_::NF; i += blockDim.x) S.fm[i] = fmask_g[i];
  if (tid == 0) {
    mbar_init(smem_u32(S.bar), 1);
    if (C_::STAGE) mbar_init(smem_u32(S.st_bar), 1);
    *S.abort = 0;
  }
  if (tid < 32) tmem_alloc(smem_u32(S.tmem), C_::TMEM_COLS);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// Per-block pipeline state: MMA and staging mbarrier parities, and whether a staging copy has
// been issued and not yet waited for.
struct Pipe {
  uint32_t phase = 0, sphase = 0;
  bool staged = false;
};

template <class C_>
__device__ __forceinline__ void block_teardown(const Smem<C_>& S, const Pipe& p) {
  // after an abort the MMA group whose wait timed out (parity phase ^ 1) may still be in
  // flight: give it one more wait, with the full bound, before the accumulator is released.
  // The decision is a block-wide OR: a thread whose last wait ran out has set the flag itself.
  // Staging copies still in flight are waited for before the block's shared memory is released.
  if (C_::STAGE) cp_async_wait_all();
  if (__syncthreads_or(*S.abort) && threadIdx.x == 0) mbar_wait(smem_u32(S.bar), p.phase ^ 1u);
  if (C_::STAGE && p.staged && threadIdx.x == 0) mbar_wait(smem_u32(S.st_bar), p.sphase);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32) tmem_dealloc(*S.tmem, C_::TMEM_COLS);
}

// Column groups of 8 that npad accumulator columns split into among the block's warps: the most
// groups, at most max_groups, that divide npad into multiples of 8.
__host__ __device__ constexpr int copy_groups(int npad, int max_groups) {
  for (int g = max_groups; g > 1; --g)
    if (npad % (8 * g) == 0) return g;
  return 1;
}

// Issue the MMAs of chunk c (width/16 k-steps x 6 split products) and commit them to the
// mbarrier.  Chunks 0 .. NVOL-1 are KV columns wide, the surface chunks after them KS.
template <class C_>
__device__ __forceinline__ void issue_chunk(const Smem<C_>& S, int c) {
  const uint32_t a0 = smem_u32(S.A), b0 = smem_u32(S.B), tmem = *S.tmem;
  // products (A term, B term) whose term orders add up to at most 2
  constexpr int PA[6] = {0, 0, 1, 0, 1, 2}, PB[6] = {0, 1, 0, 2, 1, 0};
  const bool vol = c < C_::NVOL;
  const int nks = (vol ? C_::KV : C_::KS) / 16;
  const int col8 = (vol ? c * C_::KV : C_::NVOL * C_::KV + (c - C_::NVOL) * C_::KS) / 8;  // first column / 8
#pragma unroll
  for (int ks = 0; ks < C_::KA / 16; ++ks) {
    if (ks >= nks) break;
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      const uint64_t ad = umma_desc(a0 + PA[p] * C_::A_TERM + ks * 2 * C_::A_LBO, C_::A_LBO, C_::A_SBO);
      const uint64_t bd = umma_desc(b0 + PB[p] * C_::B_TERM + (col8 + 2 * ks) * C_::B_LBO, C_::B_LBO, C_::B_SBO);
      mma_bf16(tmem, ad, bd, C_::IDESC, (c > 0 || ks > 0 || p > 0) ? 1u : 0u);
    }
  }
  mma_commit(smem_u32(S.bar));
}

// After a chunk's operand is in the slot: make it visible to the tensor core, issue its MMAs
// and wait for them (the slot is rewritten next).  Returns false once any wait has timed out
// (uniform across the block).
// The stop decision is a block-wide OR of the flag as each thread sees it on arrival: a thread whose
// wait ran out wrote the flag before arriving, so every thread gets the same answer even when
// another thread reads the flag before that write.  `polls` bounds each wait (0: the default).
// `during()` runs between the issue and the wait (loads that overlap the MMAs).
struct Nothing {
  __device__ void operator()() const {}
};

template <class C_, class During = Nothing>
__device__ __forceinline__ bool run_chunk(const Smem<C_>& S, int c, uint32_t& phase, unsigned* status,
                                          int polls = 0, const During& during = During()) {
  fence_async_smem();
  tc_fence_before();
  if (__syncthreads_or(*S.abort)) return false;
  if (threadIdx.x == 0) {
    tc_fence_after();
    issue_chunk<C_>(S, c);
  }
  during();
  if (!mbar_wait(smem_u32(S.bar), phase, polls > 0 ? polls : kWaitPolls)) {
    *S.abort = 1;
    atomicOr(status, (unsigned)DG_STATUS_TIMEOUT);
  }
  phase ^= 1u;
  tc_fence_after();
  return true;
}

// A tile's geometric factors and (C_::VM) neighbour map into shared memory by asynchronous
// copies, whose latency overlaps the node loads issued after them; the caller completes them
// (cp_async_wait_all) before the barrier that publishes them.
template <class C_>
__device__ __forceinline__ void stage_tile_tables(const Smem<C_>& S, const MixedCase& c, int e0, int nel) {
  static_assert(C_::NF % 4 == 0, "whole 16 B rows of the neighbour map (NF = 4 Nfp, row starts 16 B aligned)");
  const float* gs = c.geo + (size_t)e0 * GS;
  for (int i = threadIdx.x; i < nel * GS; i += C_::NT) cp_async4(S.geo + i, gs + i);
  if constexpr (C_::VM) {
    const int4* vs = reinterpret_cast<const int4*>(c.vmapP + (size_t)e0 * C_::NF);
    int4* vd = reinterpret_cast<int4*>(S.vm);
    for (int i = threadIdx.x; i < nel * (C_::NF / 4); i += C_::NT) cp_async16(vd + i, vs + i);
  }
}

// Issue the staging copies of tile [e0, e0 + 25) of case c (C_::STAGE): node records and, for
// Navier-Stokes, viscous-flux records by the TMA engine (thread 0; completion on st_bar), the Q_z
// values, geometric factors and neighbour map by per-thread asynchronous copies (each thread's
// cp_async_wait_all; thread t copies the Q_z values of the nodes it reads in the flux phase).
template <class C_, bool NS>
__device__ __forceinline__ void stage_issue(const Smem<C_>& S, const MixedCase& c, int e0) {
  const int nel = min(C_::E, c.K - e0), nn = nel * C_::Np;
  const size_t base = (size_t)e0 * C_::Np;
  if (threadIdx.x == 0) {
    const uint32_t bar = smem_u32(S.st_bar);
    mbar_expect_tx(bar, (uint32_t)nn * (NS ? 64u : 32u));
    bulk_g2s(S.st_node, c.node + 2 * base, (uint32_t)nn * 32u, bar);
    if (NS) bulk_g2s(S.st_fv4, c.fv4 + 2 * base, (uint32_t)nn * 32u, bar);
  }
  if (NS)
    for (int i = threadIdx.x; i < nn; i += C_::NT) cp_async4(S.st_fvz + i, c.fvz + base + i);
  stage_tile_tables<C_>(S, c, e0, nel);
}

// Neighbour-map entry of face node mm of tile element e: from the staged copy where there is one.
template <class C_>
__device__ __forceinline__ int tile_vmap(const Smem<C_>& S, const MixedCase& c, int e0, int e, int mm) {
  if constexpr (C_::VM) return S.vm[e * C_::NF + mm];
  return c.vmapP[(size_t)(e0 + e) * C_::NF + mm];
}

// Elements [e0, e0 + 25) of case c: right-hand side (RK = false: out = rhs) or the LSRK stage
// (k <- a k + dt rhs, out <- qin + b k).  Returns false when the block must stop (timeout).
// A mixture node's float state (13 values, absent species 0) from its record; returns p_hi.
__device__ __forceinline__ float load_mix_record(const float4* r, float* q) {
  const float4 a = r[0], b = r[1], c = r[2], d = r[3];
  q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w; q[4] = b.x;
  q[5] = c.x; q[6] = c.y; q[7] = c.z; q[8] = c.w;
  q[9] = d.x; q[10] = d.y; q[11] = d.z; q[12] = d.w;
  return b.y;
}

template <class C_, int PHYS, bool RK>
__device__ __forceinline__ bool rhs_tile(const Smem<C_>& S, const MixedCase& c, const double* __restrict__ qin,
                                         double* __restrict__ out, const int e0, const double a, const double b,
                                         Pipe& p, unsigned* status, const MixedCase* next, int next_e0) {
  constexpr int Np = C_::Np, Nfp = C_::Nfp, NF = C_::NF, KV = C_::KV, NT = C_::NT, NPT = C_::NPT, V = C_::V;
  constexpr bool NS = tile_ns(PHYS), MIX = PHYS == kern::MIXTURE, AVP = kern::has_av(PHYS);
  constexpr bool ST = C_::STAGE && !MIX;  // own records staged in shared memory
  static_assert(MIX ? V == mixk::MIX_V : V == 5, "5 conserved variables, or the 13 of a mixture record");
  const int tid = threadIdx.x;
  const int nvar = MIX ? c.nvar : 5;
  const int nel = min(C_::E, c.K - e0);
  const int nn = nel * Np;
  const size_t KNp = (size_t)c.K * Np;
  const size_t base = (size_t)e0 * Np;

  if (tid == 0) {
    // this tile's RK inputs (read only in the epilogue) and the next tile's inputs, into L2
    if (RK)
      for (int v = 0; v < nvar; ++v) {
        if (a != 0.0) prefetch_l2(c.k + v * KNp + base, (size_t)nn * 8);
        prefetch_l2(qin + v * KNp + base, (size_t)nn * 8);
      }
    if (next) {
      const int nnel = min(C_::E, next->K - next_e0);
      prefetch_tile_inputs(*next, next_e0, nnel, Np, NF, MIX, NS);
    }
  }
  if constexpr (ST) {
    // this tile's staged records, copied during the previous tile (or the block set-up)
    cp_async_wait_all();
    if (mbar_wait(smem_u32(S.st_bar), p.sphase, c.wait_polls > 0 ? c.wait_polls : kWaitPolls)) {
      p.sphase ^= 1u;
      p.staged = false;
    } else {  // the tile is abandoned at the first MMA round (block-wide OR of the flag)
      *S.abort = 1;
      atomicOr(status, (unsigned)DG_STATUS_TIMEOUT);
    }
  } else {
    stage_tile_tables<C_>(S, c, e0, nel);
  }
  // the tile's own node records (tile-local node index), staged or in global memory
  const float4* ND = ST ? S.st_node : c.node + 2 * base;
  const float4* FV4 = ST ? S.st_fv4 : c.fv4 + 2 * base;
  const float* FVZ = ST ? S.st_fvz : c.fvz + base;

  // volume fluxes of this thread's nodes (FP32; pressure relative to the element's first node in FP64)
  float F[NPT][3][V];
#pragma unroll
  for (int s = 0; s < NPT; ++s) {
    const int n = tid + s * NT;
    if (n < nn) {
      const int e = n / Np;
      const size_t gn = base + n, g1 = base + (size_t)e * Np;
      if constexpr (MIX) {
        float qv[V];
        const float4 ref = c.mrec[4 * g1 + 1];
        const float p1 = load_mix_record(c.mrec + 4 * gn, qv);
        const float p_lo = c.mrec[4 * gn + 1].z;
        mixk::node_flux_mix<V>(qv, nvar, (p1 - ref.y) + (p_lo - ref.z), p1, F[s]);
      } else {
        const int l1 = e * Np;
        const float4 a0 = ND[2 * n], a1 = ND[2 * n + 1], r1 = ND[2 * l1 + 1];
        const float qv[5] = {a0.x, a0.y, a0.z, a0.w, a1.x};
        float fv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if constexpr (NS) {
          const float4 f0 = FV4[2 * n], f1 = FV4[2 * n + 1];
          fv[0] = f0.x; fv[1] = f0.y; fv[2] = f0.z; fv[3] = f0.w;
          fv[4] = f1.x; fv[5] = f1.y; fv[6] = f1.z; fv[7] = f1.w;
          fv[8] = FVZ[n];
        }
        // p - p_1 from the hi/lo pairs; p itself (energy flux) as its FP32 rounding
        mixk::node_flux<NS>(qv, (a1.y - r1.y) + (a1.z - r1.z), a1.y, fv, F[s]);
        if constexpr (AVP) {  // minus the artificial-viscosity flux, where the element has eps > 0
          if (c.av_eps[e0 + e] > 0.0) {
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
              for (int v = 0; v < 5; ++v) F[s][d][v] -= cvt::narrow(c.av_sig[(5 * d + v) * KNp + gn]);
          }
        }
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();  // geometry in place; the previous tile's accumulator copy has been cleared

  // three volume chunks: contravariant flux sum_d (dr_a/dx_d) F_d at column i
#pragma unroll
  for (int ra = 0; ra < 3; ++ra) {
#pragma unroll
    for (int s = 0; s < NPT; ++s) {
      const int n = tid + s * NT;
      if (n < nn) {
        const int e = n / Np, i = n - e * Np;
        const float* G = S.geo + e * GS;
        const float gx = G[3 * ra], gy = G[3 * ra + 1], gz = G[3 * ra + 2];
#pragma unroll
        for (int v = 0; v < V; ++v)
          put3_umma(S.A, C_::A_TERM, umma_off(e * V + v, i, C_::A_LBO, C_::A_SBO),
                    fmaf(gx, F[s][0][v], fmaf(gy, F[s][1][v], gz * F[s][2][v])));
      }
    }
    if (!run_chunk<C_>(S, ra, p.phase, status, c.wait_polls)) return false;
  }

  // surface chunks: face nodes [sc KS, sc KS + KS) of every element
  const float gam = (float)c.gas.gamma;
#pragma unroll 1
  for (int sc = 0; sc < C_::NSURF; ++sc) {
    const int m0 = sc * C_::KS, w = min(C_::KS, NF - m0);
    for (int j = tid; j < nel * w; j += NT) {
      const int e = j / w, mm = m0 + (j - e * w), f = mm / Nfp;
      const float* G = S.geo + e * GS;
      const float n3[3] = {G[9 + 4 * f], G[10 + 4 * f], G[11 + 4 * f]};
      const float fs = G[12 + 4 * f];
      const int ownl = e * Np + S.fm[mm];
      const size_t own = base + ownl;
      const int Pi = tile_vmap<C_>(S, c, e0, e, mm);  // < 0: boundary face node, -DG_BC_* code
      const size_t P = Pi >= 0 ? (size_t)Pi : own;     // a boundary node gathers its own record
      const size_t Pl = P - base;                      // tile-local index (wraps when P < base)
      const bool Pin = ST && Pl < (size_t)nn;          // the neighbour's records are staged too
      float g[V];
      if constexpr (MIX) {
        float qm[V], qp[V];
        const float4 am = c.mrec[4 * own + 1];  // {rho E, p_hi, p_lo, c}
        float4 ap = c.mrec[4 * P + 1];
        load_mix_record(c.mrec + 4 * own, qm);
        load_mix_record(c.mrec + 4 * P, qp);
        const float4 lm = c.mlo[own];
        float4 lp = c.mlo[P];
        if (Pi < 0) mixk::ghost_mix_record(-Pi, n3, c, qp, ap, lp);
        const float dlo[4] = {lm.x - lp.x, lm.y - lp.y, lm.z - lp.z, lm.w - lp.w};
        mixk::face_term_mix<V>(qm, qp, nvar, am.y, ap.y, (am.y - ap.y) + (am.z - ap.z), am.w, ap.w, n3, dlo, g);
      } else {
        const float4 m0r = ND[2 * ownl], m1r = ND[2 * ownl + 1];
        float4 p0r = Pin ? S.st_node[2 * Pl] : c.node[2 * P], p1r = Pin ? S.st_node[2 * Pl + 1] : c.node[2 * P + 1];
        if (Pi < 0) mixk::ghost_record(-Pi, n3, c, p0r, p1r);
        const float qm[5] = {m0r.x, m0r.y, m0r.z, m0r.w, m1r.x}, qp[5] = {p0r.x, p0r.y, p0r.z, p0r.w, p1r.x};
        const float dpn = (m1r.y - p1r.y) + (m1r.z - p1r.z);  // p- - p+ from the hi/lo pairs
        float fvm[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, fvp[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if constexpr (NS) {
          const float4 a = FV4[2 * ownl], b2 = FV4[2 * ownl + 1];
          const float4 cc4 = Pin ? S.st_fv4[2 * Pl] : c.fv4[2 * P], d4 = Pin ? S.st_fv4[2 * Pl + 1] : c.fv4[2 * P + 1];
          fvm[0] = a.x; fvm[1] = a.y; fvm[2] = a.z; fvm[3] = a.w;
          fvm[4] = b2.x; fvm[5] = b2.y; fvm[6] = b2.z; fvm[7] = b2.w; fvm[8] = FVZ[ownl];
          fvp[0] = cc4.x; fvp[1] = cc4.y; fvp[2] = cc4.z; fvp[3] = cc4.w;
          fvp[4] = d4.x; fvp[5] = d4.y; fvp[6] = d4.z; fvp[7] = d4.w; fvp[8] = Pin ? S.st_fvz[Pl] : c.fvz[P];
          if (Pi < 0) mixk::ghost_viscous(-Pi, n3, fvp);
        }
        mixk::face_term<NS>(qm, qp, m1r.y, p1r.y, dpn, fvm, fvp, n3, gam, g);
        if constexpr (AVP) {
          // central artificial-viscosity flux: g gains -(n.sigma- - n.sigma+)/2; at a boundary node
          // P is the node itself, so the term vanishes (sigma+ = sigma-)
          const bool onM = c.av_eps[e0 + e] > 0.0, onP = c.av_eps[P / Np] > 0.0;
          if (onM || onP) {
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              double sm = 0.0, sp = 0.0;
              if (onM)
                sm = fma((double)n3[0], c.av_sig[v * KNp + own],
                         fma((double)n3[1], c.av_sig[(5 + v) * KNp + own], (double)n3[2] * c.av_sig[(10 + v) * KNp + own]));
              if (onP)
                sp = fma((double)n3[0], c.av_sig[v * KNp + P],
                         fma((double)n3[1], c.av_sig[(5 + v) * KNp + P], (double)n3[2] * c.av_sig[(10 + v) * KNp + P]));
              g[v] -= 0.5f * cvt::narrow(sm - sp);
            }
          }
        }
      }
#pragma unroll
      for (int v = 0; v < V; ++v)
        put3_umma(S.A, C_::A_TERM, umma_off(e * V + v, mm - m0, C_::A_LBO, C_::A_SBO), fs * g[v]);
    }
    if (sc < C_::NSURF - 1) {
      if (!run_chunk<C_>(S, 3 + sc, p.phase, status, c.wait_polls)) return false;
    }
  }
  // the last surface chunk; this thread's RK inputs are loaded while its MMAs run
  double k_old[NPT][V], q_old[NPT][V];
  const auto load_rk = [&] {
#pragma unroll
    for (int s = 0; s < NPT; ++s) {
      const int n = tid + s * NT;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const size_t gi = v * KNp + base + n;
        k_old[s][v] = (RK && n < nn && v < nvar && a != 0.0) ? c.k[gi] : 0.0;
        q_old[s][v] = (RK && n < nn && v < nvar) ? qin[gi] : 0.0;
      }
    }
  };
  // every thread is past its reads of the staged records: the next tile's copies start now
  const auto during = [&] {
    if constexpr (ST) {
      if (next) {
        stage_issue<C_, NS>(S, *next, next_e0);
        p.staged = true;
      }
    }
    load_rk();
  };
  if (!run_chunk<C_>(S, 3 + C_::NSURF - 1, p.phase, status, c.wait_polls, during)) return false;

  // accumulator -> shared memory (warps 0..3 own TMEM lanes 0..127), then the node-parallel update
  if (tid < 128) {
    const int warp = tid >> 5, row = tid;
    float* Crow = S.C + row * C_::CS;
#pragma unroll
    for (int c0 = 0; c0 < C_::NPAD; c0 += 16) {
      float r[16];
      tmem_ld16(*S.tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
#pragma unroll
      for (int j = 0; j < 16; ++j) Crow[c0 + j] = r[j];
    }
  }
  tc_fence_before();
  __syncthreads();
  const float dtf = (float)c.dt;
#pragma unroll
  for (int s = 0; s < NPT; ++s) {
    const int n = tid + s * NT;
    if (n < nn) {
      const int e = n / Np, i = n - e * Np;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        if (v < nvar) {
          const float r = S.C[(e * V + v) * C_::CS + i];
          const size_t gi = v * KNp + base + n;
          if (RK) {
            // dt rhs formed in FP32 (the right-hand side carries FP32-level error already) and
            // widened on the integer pipe; the accumulation is FP64
            const double kk = fma(a, k_old[s][v], cvt::widen(dtf * r));
            c.k[gi] = kk;
            out[gi] = fma(b, kk, q_old[s][v]);
          } else {
            out[gi] = cvt::widen(r);
          }
        }
      }
    }
  }
  // the accumulator copy overwrote operand columns that no chunk rewrites (padding whose
  // operator entries are zero): clear it, so that they hold zeros rather than FP32 bit
  // patterns read as BF16 (possibly NaN, and 0 x NaN = NaN)
  __syncthreads();
  uint4* Cz = reinterpret_cast<uint4*>(S.C);
  for (int i = tid; i < C_::ROWS * C_::CS / 4; i += NT) Cz[i] = make_uint4(0u, 0u, 0u, 0u);
  return true;
}

// ---- kernels ---------------------------------------------------------------------------------
// Variables per element row block: 5, or 5 + DG_MAX_SPECIES for a mixture.
__host__ __device__ constexpr int tile_v(int PHYS) { return PHYS == kern::MIXTURE ? mixk::MIX_V : 5; }

template <int N, int NT, int PHYS, bool RK>
__global__ void __launch_bounds__(NT, (Cfg<N, NT, tile_v(PHYS)>::MINB)) rhs_tc_kernel(const MixedCase c, const uint4* __restrict__ b_g,
                                                             const int32_t* __restrict__ fmask_g, const double a,
                                                             const double b, unsigned* __restrict__ status) {
  using C_ = Cfg<N, NT, tile_v(PHYS)>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const Smem<C_> S(smem_raw);
  block_setup<C_>(S, b_g, fmask_g);
  Pipe p;
  if constexpr (C_::STAGE && PHYS != kern::MIXTURE) {
    if (blockIdx.x * C_::E < c.K) {
      stage_issue<C_, tile_ns(PHYS)>(S, c, blockIdx.x * C_::E);
      p.staged = true;
    }
  }
  for (int e0 = blockIdx.x * C_::E; e0 < c.K; e0 += gridDim.x * C_::E) {
    const int ne0 = e0 + gridDim.x * C_::E;
    if (!rhs_tile<C_, PHYS, RK>(S, c, c.q[0], c.q[1], e0, a, b, p, status, ne0 < c.K ? &c : nullptr, ne0))
      break;
  }
  block_teardown<C_>(S, p);
}

// A batch of cases: persistent over a work list of (case, first element) tiles; the stage's
// parity picks input and output among each case's two state buffers.
template <int N, int NT, int PHYS>
__global__ void __launch_bounds__(NT, (Cfg<N, NT>::MINB)) rhs_tc_batched(const MixedCase* __restrict__ cases,
                                                              const int2* __restrict__ work, const int nwork,
                                                              const uint4* __restrict__ b_g,
                                                              const int32_t* __restrict__ fmask_g, const int stage,
                                                              const double a, const double b,
                                                              unsigned* __restrict__ status) {
  using C_ = Cfg<N, NT>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const Smem<C_> S(smem_raw);
  block_setup<C_>(S, b_g, fmask_g);
  Pipe p;
  if constexpr (C_::STAGE && PHYS != kern::MIXTURE) {
    if (blockIdx.x < nwork) {
      const int2 it = work[blockIdx.x];
      stage_issue<C_, tile_ns(PHYS)>(S, cases[it.x], it.y);
      p.staged = true;
    }
  }
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 it = work[w];
    const MixedCase& c = cases[it.x];
    const int wn = w + gridDim.x;
    const int2 nx = wn < nwork ? work[wn] : make_int2(0, 0);
    if (!rhs_tile<C_, PHYS, true>(S, c, c.q[stage & 1], c.q[(stage & 1) ^ 1], it.y, a, b, p, status,
                                  wn < nwork ? &cases[nx.x] : nullptr, nx.y))
      break;
  }
  block_teardown<C_>(S, p);
}

// Issue the staging copies of BR1 tile [e0, e0 + 25) of case c (C_::STAGE): node records and
// temperature pairs by the TMA engine (thread 0; completion on st_bar).
// With odd Np the temperature pairs go by per-thread 8-byte asynchronous copies instead, thread t
// copying those of the nodes t + j NT that it reads itself (each thread completes its copies with
// cp_async_wait_all before it reads them).
template <class C_>
__device__ __forceinline__ void stage_issue_vis(const Smem<C_>& S, const MixedCase& c, int e0) {
  const int nel = min(C_::E, c.K - e0), nn = nel * C_::Np;
  const size_t base = (size_t)e0 * C_::Np;
  if (threadIdx.x == 0) {
    const uint32_t bar = smem_u32(S.st_bar);
    mbar_expect_tx(bar, (uint32_t)nn * (C_::TEMP_BULK ? 40u : 32u));
    bulk_g2s(S.st_node, c.node + 2 * base, (uint32_t)nn * 32u, bar);
    if (C_::TEMP_BULK) bulk_g2s(S.st_temp, c.temp + base, (uint32_t)nn * 8u, bar);
  }
  if (!C_::TEMP_BULK)
    for (int i = threadIdx.x; i < nn; i += C_::NT) cp_async8(S.st_temp + i, c.temp + base + i);
}

// ==== BR1 pass on the tensor cores ===============================================================
// For affine tetrahedra the outward normal times Fscale of face f is a fixed combination of the
// rows of dr/dx (Nanson's relation): n_f Fscale_f = sum_a c_{f,a} grad r_a with c = (0,0,-1),
// (0,-1,0), (1,1,1), (-1,0,0) for faces 0..3.  The lifted central-flux jump of BR1 therefore
// folds into element-independent operators:
//   grad_d w = sum_a (dr_a/dx_d) ( D_a w + Lhat_a jump ),  Lhat_a = 1/2 sum_f c_{f,a} LIFT_f,
// with jump = w+ - w- at the face nodes.  One contraction of [w | jump] (rows (element, field))
// against [D_a | Lhat_a] for a = r, s, t (N = 3 NPAD output columns) gives the three reference
// derivatives; the geometric factors and the stress follow per node.
template <int N, int NT_ = default_vis_nt(N)>
struct VCfg {
  using O = kern::Ord<N>;
  static constexpr int ORDER = N;
  static constexpr int Np = O::Np, Nfp = O::Nfp, NF = O::NF;
  static constexpr int E = 25, ROWS = 128;
  static constexpr int KV = round16(Np), NPAD = KV, NOUT = 3 * NPAD;
  static constexpr int NVOL = 1, KS = surface_cols(N, KV, NF), KA = KS > KV ? KS : KV;
  static constexpr int NSURF = (NF + KS - 1) / KS, NCHUNK = NVOL + NSURF, KB = NVOL * KV + NSURF * KS;
  static constexpr int A_LBO = 144, A_SBO = (KA / 8) * A_LBO, A_TERM = 16 * A_SBO;
  static constexpr int B_LBO = 128, B_SBO = (KB / 8) * B_LBO, B_TERM = (NOUT / 8) * B_SBO;
  static constexpr int CS = NPAD + 1;  // one reference direction's columns are copied at a time
  static constexpr int TMEM_COLS = NOUT <= 64 ? 64 : (NOUT <= 128 ? 128 : 256);
  static constexpr int NT = NT_;
  static constexpr int NODES = E * Np, NPT = (NODES + NT - 1) / NT;
  static constexpr uint32_t IDESC = idesc_bf16(ROWS, NOUT);
  static constexpr int OFF_B = 0, OFF_A = 3 * B_TERM, OFF_GEO = OFF_A + 3 * A_TERM;
  static constexpr int OFF_FM = OFF_GEO + E * GS * 4;
  static constexpr int OFF_VM = (OFF_FM + NF * 4 + 15) / 16 * 16, VM_BYTES = E * NF * 4;
  static constexpr bool VM = vm_fits(OFF_FM + NF * 4, OFF_VM + VM_BYTES, NT, 64);
  static constexpr int END_VM = VM ? OFF_VM + VM_BYTES : OFF_FM + NF * 4;
  // the tile's own node records and temperature pairs, staged one tile ahead where that costs no
  // resident block: [E Np] x 2 float4 by a bulk copy, [E Np] float2 by one too for even Np (tile
  // starts and sizes are then 16-byte multiples), else by per-thread asynchronous copies
  static constexpr int OFF_ST = (END_VM + 15) / 16 * 16, ST_BYTES = E * Np * 40;
  static constexpr bool STAGE = VM && vm_fits(END_VM, OFF_ST + ST_BYTES, NT, 64);
  static constexpr bool TEMP_BULK = Np % 2 == 0;
  static constexpr int OFF_BAR = ((STAGE ? OFF_ST + ST_BYTES : END_VM) + 7) / 8 * 8;
  static constexpr int SMEM = OFF_BAR + 24;
  static constexpr int MINB = aim_blocks(SMEM, NT);
  static_assert(NT % 32 == 0 && NT >= 128 && NT <= 1024, "whole warps, at least the four TMEM lane quarters");
  static_assert(NOUT <= 256 && NOUT % 16 == 0, "MMA N");
  static_assert(ROWS * CS * 4 <= 3 * A_TERM && ROWS * CS % 4 == 0, "accumulator copy in the operand slot");
  static_assert(NOUT <= TMEM_COLS, "TMEM columns");
  // Row-parallel gradients (where they fit in the operand slot): the threads of an accumulator row
  // (element, field) read the row from TMEM for the three reference directions at once and write
  // the node gradients [E Np][3][5] (stride GSTR floats per node) to shared memory; the warps
  // split the columns into CG groups of 8 (warp w: TMEM lane quarter w % 4, group w / 4).
  static constexpr int GSTR = 15, CG = copy_groups(NPAD, NT / 128), CPG = NPAD / CG;
  static constexpr bool ROWGRAD = E * Np * GSTR * 4 <= 3 * A_TERM && CPG % 8 == 0;
  static constexpr int CLEAR_BYTES = ROWGRAD ? (E * Np * GSTR * 4 + 15) / 16 * 16 : ROWS * CS * 4;
};

// Elements [e0, e0 + 25) of case c: the viscous-flux records from the node records (rho and T as
// hi/lo pairs, momentum) and the temperature pairs.
template <class C_>
__device__ __forceinline__ bool vis_tile(const Smem<C_>& S, const MixedCase& c, const int e0, Pipe& p,
                                         unsigned* status, const MixedCase* next, int next_e0) {
  constexpr int Np = C_::Np, NF = C_::NF, KV = C_::KV, NT = C_::NT, NPT = C_::NPT;
  constexpr bool ST = C_::STAGE;
  const int tid = threadIdx.x;
  const int nel = min(C_::E, c.K - e0);
  const int nn = nel * Np;
  const size_t KNp = (size_t)c.K * Np;
  const size_t base = (size_t)e0 * Np;

  if (tid == 0 && next) {
    // the next tile's inputs into L2: node records, temperature pairs, geometry, neighbour map
    const int nnel = min(C_::E, next->K - next_e0);
    const size_t nb = (size_t)next_e0 * Np, nnn = (size_t)nnel * Np;
    prefetch_l2(next->node + 2 * nb, nnn * 32);
    prefetch_l2(next->temp + nb, nnn * 8);
    prefetch_l2(next->geo + (size_t)next_e0 * GS, (size_t)nnel * GS * 4);
    prefetch_l2(next->vmapP + (size_t)next_e0 * NF, (size_t)nnel * NF * 4);
  }
  if constexpr (ST) {
    // this tile's staged records, copied during the previous tile (or the block set-up); the
    // only asynchronous copies of this thread in flight here are its temperature pairs (odd Np)
    if (!C_::TEMP_BULK) cp_async_wait_all();
    if (mbar_wait(smem_u32(S.st_bar), p.sphase, c.wait_polls > 0 ? c.wait_polls : kWaitPolls)) {
      p.sphase ^= 1u;
      p.staged = false;
    } else {  // the tile is abandoned at the first MMA round (block-wide OR of the flag)
      *S.abort = 1;
      atomicOr(status, (unsigned)DG_STATUS_TIMEOUT);
    }
  }
  stage_tile_tables<C_>(S, c, e0, nel);
  // the tile's own node records and temperature pairs (tile-local node index)
  const float4* ND = ST ? S.st_node : c.node + 2 * base;
  const float2* TD = ST ? S.st_temp : c.temp + base;

  // volume chunk: (rho - rho_1, m, T - T_1) per node; the differences to the element's first node
  // from the hi/lo pairs
  float rho_n[NPT], m_n[NPT][3], w_n[NPT][5];
#pragma unroll
  for (int s = 0; s < NPT; ++s) {
    const int n = tid + s * NT;
    if (n < nn) {
      const int l1 = (n / Np) * Np;
      const float4 a0 = ND[2 * n], a1 = ND[2 * n + 1];
      const float4 r0 = ND[2 * l1], r1 = ND[2 * l1 + 1];
      // (with per-thread temperature copies the reference node's pair is another thread's: global)
      const float2 t = TD[n], t1 = (ST && !C_::TEMP_BULK) ? c.temp[base + l1] : TD[l1];
      rho_n[s] = a0.x;
      m_n[s][0] = a0.y;
      m_n[s][1] = a0.z;
      m_n[s][2] = a0.w;
      w_n[s][0] = (a0.x - r0.x) + (a1.w - r1.w);
      w_n[s][1] = a0.y;
      w_n[s][2] = a0.z;
      w_n[s][3] = a0.w;
      w_n[s][4] = (t.x - t1.x) + (t.y - t1.y);
    }
  }
  cp_async_wait_all();
  __syncthreads();  // geometry in place; the previous tile's accumulator copy has been cleared
#pragma unroll
  for (int s = 0; s < NPT; ++s) {
    const int n = tid + s * NT;
    if (n < nn) {
      const int e = n / Np, i = n - e * Np;
#pragma unroll
      for (int f = 0; f < 5; ++f)
        put3_umma(S.A, C_::A_TERM, umma_off(e * 5 + f, i, C_::A_LBO, C_::A_SBO), w_n[s][f]);
    }
  }
  if (!run_chunk<C_>(S, 0, p.phase, status, c.wait_polls)) return false;

  // surface chunks: jumps w+ - w- at face nodes [sc KS, sc KS + KS)
#pragma unroll 1
  for (int sc = 0; sc < C_::NSURF; ++sc) {
    const int m0 = sc * C_::KS, w = min(C_::KS, NF - m0);
    for (int j = tid; j < nel * w; j += NT) {
      const int e = j / w, mm = m0 + (j - e * w);
      const int ownl = e * Np + S.fm[mm];
      const int Pi = tile_vmap<C_>(S, c, e0, e, mm);    // < 0: boundary face node, -DG_BC_* code
      const size_t P = Pi >= 0 ? (size_t)Pi : base + ownl;  // a boundary node gathers its own record
      const size_t Pl = P - base;                           // tile-local index (wraps when P < base)
      const bool Pin = ST && Pl < (size_t)nn;               // the neighbour's records are staged too
      const float4 o0 = ND[2 * ownl], o1 = ND[2 * ownl + 1];
      const float4* pn = Pin ? S.st_node + 2 * Pl : c.node + 2 * P;
      float4 q0 = pn[0], q1 = pn[1];
      const float2 to = TD[ownl];
      float2 tp = Pin ? S.st_temp[Pl] : c.temp[P];
      if (Pi < 0) {  // exterior values w(q+) of the face's ghost state
        const int f = mm / C_::Nfp;
        const float* G = S.geo + e * GS;
        const float n3[3] = {G[9 + 4 * f], G[10 + 4 * f], G[11 + 4 * f]};
        mixk::ghost_record(-Pi, n3, c, q0, q1);
        if (-Pi == DG_BC_INFLOW) tp = c.in_temp;
      }
      const float jv[5] = {(q0.x - o0.x) + (q1.w - o1.w), q0.y - o0.y, q0.z - o0.z, q0.w - o0.w,
                           (tp.x - to.x) + (tp.y - to.y)};
#pragma unroll
      for (int f = 0; f < 5; ++f)
        put3_umma(S.A, C_::A_TERM, umma_off(e * 5 + f, mm - m0, C_::A_LBO, C_::A_SBO), jv[f]);
    }
    // after the last gathers every thread is past its reads of the staged records: the next
    // tile's copies start with the MMAs (the staged node records are not read again here)
    const auto during = [&] {
      if constexpr (ST) {
        if (sc == C_::NSURF - 1 && next) {
          stage_issue_vis<C_>(S, *next, next_e0);
          p.staged = true;
        }
      }
    };
    if (!run_chunk<C_>(S, 1 + sc, p.phase, status, c.wait_polls, during)) return false;
  }

  const float mu = (float)c.gas.mu, kap = (float)c.gas.kappa;
  if constexpr (C_::ROWGRAD) {
    // reference derivatives -> gradients, row-parallel: accumulator row r = 5 e + f holds
    // D_a w_f + Lhat_a [w_f] of tile element e at columns a NPAD + i; the threads of the row (TMEM
    // lane quarter r / 32, one column group each) form grad_d w_f = sum_a (dr_a/dx_d)(...) at their
    // nodes and write them to the buffer [E Np][3][5], which aliases the operand slot
    float* GR = S.C;
    const int warp = tid >> 5, lane = tid & 31;
    if (warp < 4 * C_::CG) {
      const int q = warp & 3, g = warp >> 2, r = 32 * q + lane;
      const int e = r / 5, f = r - 5 * e;
      const bool row_ok = e < nel;  // rows past the tile's elements (and 125..127) hold nothing
      float Gm[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d) Gm[a][d] = row_ok ? S.geo[e * GS + 3 * a + d] : 0.0f;
      const uint32_t tl = *S.tmem + ((uint32_t)(32 * q) << 16);
#pragma unroll
      for (int c0 = 0; c0 < C_::CPG; c0 += 8) {
        const int col = g * C_::CPG + c0;
        float da[3][8];
#pragma unroll
        for (int a = 0; a < 3; ++a) tmem_ld8(tl + (uint32_t)(a * C_::NPAD + col), da[a]);  // the whole warp
        if (row_ok) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int i = col + jj;
            if (i < Np) {
              float* out = GR + (e * Np + i) * C_::GSTR + f;
#pragma unroll
              for (int d = 0; d < 3; ++d)  // the direction order of the per-direction form below
                out[5 * d] = fmaf(Gm[2][d], da[2][jj], fmaf(Gm[1][d], da[1][jj], fmaf(Gm[0][d], da[0][jj], 0.0f)));
            }
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
#pragma unroll
    for (int s = 0; s < NPT; ++s) {
      const int n = tid + s * NT;
      if (n < nn) {
        float grad[3][5];
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int fi = 0; fi < 5; ++fi) grad[d][fi] = GR[n * C_::GSTR + 5 * d + fi];
        float f9[9];
        mixk::viscous_flux_node(rho_n[s], m_n[s], grad, mu, kap, f9);
        const size_t gn = base + n;
        c.fv4[2 * gn] = make_float4(f9[0], f9[1], f9[2], f9[3]);
        c.fv4[2 * gn + 1] = make_float4(f9[4], f9[5], f9[6], f9[7]);
        c.fvz[gn] = f9[8];
      }
    }
    __syncthreads();  // every read of the gradient buffer is done before it is cleared
  } else {
  // reference derivatives -> gradients, one reference direction at a time through shared memory
  float grad[NPT][3][5];
#pragma unroll
  for (int s = 0; s < NPT; ++s)
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int f = 0; f < 5; ++f) grad[s][d][f] = 0.0f;
#pragma unroll 1
  for (int a = 0; a < 3; ++a) {
    // direction a's columns -> S.C, by the warps of CG column groups (warp w: TMEM lane quarter
    // w % 4, the lanes a warp may access; column group w / 4)
    if (tid < 128 * C_::CG) {
      const int warp = tid >> 5, q = warp & 3, g = warp >> 2;
      float* Crow = S.C + (32 * q + (tid & 31)) * C_::CS + g * C_::CPG;
#pragma unroll
      for (int c0 = 0; c0 < C_::CPG; c0 += 8) {
        float r[8];
        tmem_ld8(*S.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(a * C_::NPAD + g * C_::CPG + c0), r);
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) Crow[c0 + jj] = r[jj];
      }
    }
    tc_fence_before();
    __syncthreads();
#pragma unroll
    for (int s = 0; s < NPT; ++s) {
      const int n = tid + s * NT;
      if (n < nn) {
        const int e = n / Np, i = n - e * Np;
        const float* G = S.geo + e * GS + 3 * a;
#pragma unroll
        for (int f = 0; f < 5; ++f) {
          const float cv = S.C[(e * 5 + f) * C_::CS + i];
#pragma unroll
          for (int d = 0; d < 3; ++d) grad[s][d][f] = fmaf(G[d], cv, grad[s][d][f]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < NPT; ++s) {
    const int n = tid + s * NT;
    if (n < nn) {
      float f9[9];
      mixk::viscous_flux_node(rho_n[s], m_n[s], grad[s], mu, kap, f9);
      const size_t gn = base + n;
      c.fv4[2 * gn] = make_float4(f9[0], f9[1], f9[2], f9[3]);
      c.fv4[2 * gn + 1] = make_float4(f9[4], f9[5], f9[6], f9[7]);
      c.fvz[gn] = f9[8];
    }
  }
  }
  // clear what aliased the operand slot (see rhs_tile); a barrier above ordered its reads
  uint4* Cz = reinterpret_cast<uint4*>(S.C);
  for (int i = tid; i < C_::CLEAR_BYTES / 16; i += NT) Cz[i] = make_uint4(0u, 0u, 0u, 0u);
  return true;
}

template <int N, int NT>
__global__ void __launch_bounds__(NT, (VCfg<N, NT>::MINB)) vis_tc_kernel(const MixedCase c,
                                                                             const uint4* __restrict__ b_g,
                                                                             const int32_t* __restrict__ fmask_g,
                                                                             unsigned* __restrict__ status) {
  using C_ = VCfg<N, NT>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const Smem<C_> S(smem_raw);
  block_setup<C_>(S, b_g, fmask_g);
  Pipe p;
  if constexpr (C_::STAGE) {
    if (blockIdx.x * C_::E < c.K) {
      stage_issue_vis<C_>(S, c, blockIdx.x * C_::E);
      p.staged = true;
    }
  }
  for (int e0 = blockIdx.x * C_::E; e0 < c.K; e0 += gridDim.x * C_::E) {
    const int ne0 = e0 + gridDim.x * C_::E;
    if (!vis_tile<C_>(S, c, e0, p, status, ne0 < c.K ? &c : nullptr, ne0)) break;
  }
  block_teardown<C_>(S, p);
}

template <int N, int NT>
__global__ void __launch_bounds__(NT, (VCfg<N, NT>::MINB)) vis_tc_batched(const MixedCase* __restrict__ cases,
                                                                              const int2* __restrict__ work,
                                                                              const int nwork,
                                                                              const uint4* __restrict__ b_g,
                                                                              const int32_t* __restrict__ fmask_g,
                                                                              const int stage,
                                                                              unsigned* __restrict__ status) {
  using C_ = VCfg<N, NT>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const Smem<C_> S(smem_raw);
  block_setup<C_>(S, b_g, fmask_g);
  Pipe p;
  if constexpr (C_::STAGE) {
    if (blockIdx.x < nwork) {
      const int2 it = work[blockIdx.x];
      stage_issue_vis<C_>(S, cases[it.x], it.y);
      p.staged = true;
    }
  }
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 it = work[w];
    const MixedCase& c = cases[it.x];
    const int wn = w + gridDim.x;
    const int2 nx = wn < nwork ? work[wn] : make_int2(0, 0);
    if (!vis_tile<C_>(S, c, it.y, p, status, wn < nwork ? &cases[nx.x] : nullptr, nx.y)) break;
  }
  block_teardown<C_>(S, p);
}

}  // namespace tc
}  // namespace dg
