// Tensor-core variant of the mixed-precision batch tile: the three D
// contractions of the volume term (Sec. 2, Eq. (2)) as TF32 split products on
// the fifth-generation tensor cores, with FP32 accumulation in tensor memory.
//
// Contraction.  Every (direction, field) block of an element holds Nq^2 lines
// of Nq fluxes; the sweep of a line is out[i] = sum_n D[i][n] F[n].  All
// 15 blocks of a pass use the same D, so the whole stage is one product
// C = A B^T: A has a row per line (several short lines packed into one row,
// P lines of Nq values side by side), B is block-diagonal with P copies of D.
// TF32 keeps 11 significant bits, so each operand is split into a head and a
// tail: F = Fh + Fl with Fh = F with its 13 low mantissa bits cleared (what
// the tensor core reads from F itself) and Fl = F - Fh exactly, and likewise
// D = Dh + Dl.  Per 128-row block two MMAs accumulate
//   C[:, 0:H]  = Fh Dh^T + Fl Dh^T,   C[:, H:2H] = Fh Dl^T
// (B1 = [Dh; Dl] stacked along N for the head rows, B2 = [Dh; 0] for the tail
// rows), and the readback adds the two halves: F D - C = Fl Dl (2^-22 |F||D|
// relative) plus the TF32 rounding of the tails (2^-21), against the 2^-24 of
// an FP32 sweep; the mixed mode's bar is 1e-5.
//
// Layout.  A (heads and tails) and B live in shared memory in the canonical
// K-major no-swizzle layout of tcgen05.cuh: 8-row groups contiguous (SBO = 128
// bytes), K chunks of 4 values LBO = 16 ROWS + pad bytes apart.  A 4-byte
// access by a warp is free of bank conflicts when its 32 (row, slot) pairs have
// distinct (row + chunk shift) mod 8 within each class of slot mod 4; a warp of
// points that all share the coordinate along a direction (one K slot) can only
// reach 8 banks.  At Nq = 8 and 4 the thread of point (i, j, k) is chosen so
// that the two low bits of i, j and k all vary within a warp (k1 = i0 ^ j0 ^
// a warp bit), and each direction numbers its lines so that the threads of
// one slot class land on 8 distinct rows mod 8: every access of phases 1 and
// 3 is conflict-free.  Other orders keep the natural point order (about 2-way).
// Each (direction, field) block has a whole number of 8-row groups,
// so a thread's slot for field b is its field-0 slot plus b blocks (immediate
// offsets).  The readback writes each output back into the slot its flux came
// from, so phase 3 reads a point's three sweeps where phase 1 wrote its
// fluxes.  Accumulators: block m of 128 rows at TMEM columns [m 2H, (m+1) 2H).
//
// State in tensor memory.  q, dq, the nine metric terms and J^-1 of each
// point stay in TMEM for all stages (columns 160 + 24 (warp / 4) of the
// thread's lane: q 0-4, g 5-13, J^-1 14, dq 16-20), read and written with
// tcgen05.ld/st, so shared memory holds only the operands: 84.5 KB at most,
// two CTAs of 512 threads per SM, 256 TMEM columns each.
//
// Per stage: fluxes by point into A (heads and tails); one thread issues
// 2 x (row blocks) x (K steps) MMAs and commits them to an mbarrier; every
// thread waits (bounded: a wait that runs out makes the kernel report
// NUMA_ETIMEOUT through the batch's status word and stop); warps read the
// accumulators of their lane quarter back into A; points combine the three
// sweeps, scale by -J^-1, add gravity and update q and dq.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "batch_tile.cuh"
#include "eos.cuh"
#include "numa_internal.h"
#include "tcgen05.cuh"

namespace numa {

namespace {

constexpr uint32_t kTcCols = 256;        // TMEM columns per CTA
constexpr uint32_t kTcStateCol = 160;    // first column of the per-point state
constexpr uint32_t kTcStateStride = 24;  // state columns per warp of a lane quarter

__host__ __device__ constexpr int tc_round_up(int x, int m) { return (x + m - 1) / m * m; }

// Shape of the split contraction for order Nq.
template <int NQ>
struct TcShape {
    static constexpr int N3 = NQ * NQ * NQ, NL = NQ * NQ;
    static constexpr int EPP = kThreads / N3;          // elements per pass
    // lines per row: as many as fit the K steps with little padding
    static constexpr int P = NQ == 2 ? 4 : NQ == 3 ? 5 : NQ == 4 ? 2 : NQ == 5 ? 3 : NQ == 6 ? 5 : 1;
    static constexpr int PQ = P * NQ;                  // K slots a row uses
    static constexpr int KS = (PQ + 7) / 8;            // K steps of 8
    static constexpr int KW = 8 * KS;                  // K slots of a row
    static constexpr int H = KW;                       // half of the accumulator columns
    static constexpr int NN = 2 * H;                   // N of each MMA
    static constexpr int BL = tc_round_up(EPP * NL, 8 * P);   // lines per block, padded
    static constexpr int BROWS = BL / P;               // rows per block (a multiple of 8)
    static constexpr int ROWS = tc_round_up(15 * BROWS, 128);
    static constexpr int NBLK = ROWS / 128;
    // bytes between K chunks of A: ROWS 16 plus a pad that shifts the banks of
    // successive chunks (chosen per order by counting bank conflicts of the
    // phase-1 stores and phase-3 loads of every warp)
    static constexpr int PAD = NQ == 3 || NQ == 5 ? 32 : NQ == 6 ? 16 : 64;
    static constexpr int LBO_A = ROWS * 16 + PAD;
    static constexpr int REGION = 2 * KS * LBO_A;      // bytes of the heads (or the tails)
    static constexpr int LBO_B = NN * 16;
    static constexpr int BBYTES = 2 * KS * LBO_B;      // bytes of B1 (or B2)
    static constexpr int BLK_BYTES = BROWS * 16;       // bytes between (direction, field) blocks
    static constexpr int SMEM = 2 * REGION + 2 * BBYTES;
    static_assert(NBLK * NN <= (int)kTcStateCol, "accumulators overlap the state columns");
    static_assert(NN % 16 == 0 && NN <= 256, "N of an M = 128 MMA");
    static_assert(LBO_A / 16 < (1 << 14), "LBO field");
};

constexpr int tc_smem_max() {
    constexpr int s[] = {TcShape<2>::SMEM, TcShape<3>::SMEM, TcShape<4>::SMEM, TcShape<5>::SMEM,
                         TcShape<6>::SMEM, TcShape<7>::SMEM, TcShape<8>::SMEM};
    int m = 0;
    for (int x : s) m = x > m ? x : m;
    return m;
}
// Per-thread values kept in shared memory after the operands (the point's
// reference state, EOS factors and flux offsets), read where they are used so
// that they hold no registers across the stage: 8 words per thread.
constexpr int kTcAuxWords = 8;
constexpr int kTcOperandBytes = tc_smem_max();
constexpr int kTcSmemBytes = kTcOperandBytes + kTcAuxWords * kThreads * 4;
static_assert(kTcStateCol + 4 * kTcStateStride <= kTcCols, "TMEM columns");

// Head and tail of D per order (index Nq), D[i][n] at [i Nq + n]: Dh is the
// FP32 value of D with its 13 low mantissa bits cleared, Dl = D - Dh rounded
// to FP32.
struct TcDiff {
    float h[64], l[64];
};
__constant__ TcDiff c_tc_diff[9];

inline float tf32_head(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    u &= 0xFFFFE000u;
    memcpy(&x, &u, 4);
    return x;
}

inline cudaError_t upload_tc_tables() {
    TcDiff t[9] = {};
    for (int N = 1; N <= 7; ++N) {
        double D[64];
        gll_diff_matrix(N, D);
        const int nq = N + 1;
        for (int x = 0; x < nq * nq; ++x) {
            const float h = tf32_head(static_cast<float>(D[x]));
            t[nq].h[x] = h;
            t[nq].l[x] = static_cast<float>(D[x] - static_cast<double>(h));
        }
    }
    return cudaMemcpyToSymbol(c_tc_diff, t, sizeof(t));
}

__device__ __forceinline__ float tf32_head_dev(float x) {
    return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

// Byte offset of K slot s of row R in an operand with LBO `lbo`.
__device__ __forceinline__ int tc_slot(int R, int s, int lbo) {
    return (R >> 3) * 128 + (s >> 2) * lbo + (R & 7) * 16 + (s & 3) * 4;
}

// Point (el, i, j, k) of thread l.  Nq = 8 and 4: lane bits l0..l4 give
// i0, i1, j0, j1, k0 and k1 = l0 ^ l2 ^ (a warp bit); the other bits come from
// the warp index.  Other orders: l = el N3 + i + Nq j + Nq^2 k.
template <int NQ>
__device__ __forceinline__ void tc_thread_point(int l, int &el, int &i, int &j, int &k) {
    if constexpr (NQ == 8) {
        const int h = l >> 5;
        el = 0;
        i = (l & 3) | (h & 1) << 2;
        j = ((l >> 2) & 3) | ((h >> 1) & 1) << 2;
        k = ((l >> 4) & 1) | ((l ^ (l >> 2) ^ (h >> 3)) & 1) << 1 | ((h >> 2) & 1) << 2;
    } else if constexpr (NQ == 4) {
        const int h = l >> 5;
        el = h >> 1;
        i = l & 3;
        j = (l >> 2) & 3;
        k = ((l >> 4) & 1) | ((l ^ (l >> 2) ^ h) & 1) << 1;
    } else {
        constexpr int N3 = NQ * NQ * NQ;
        el = l / N3;
        const int p = l % N3;
        i = p % NQ;
        j = (p / NQ) % NQ;
        k = p / (NQ * NQ);
    }
}

// Byte offset, within a (direction, field) block, of the flux of point
// (el, i, j, k) in direction d: its line's row and its K slot.
template <int NQ>
__device__ __forceinline__ int tc_point_offset(int d, int el, int i, int j, int k) {
    using S = TcShape<NQ>;
    int line, pos;
    auto b = [](int x, int n) { return (x >> n) & 1; };
    if constexpr (NQ == 8) {   // row bits of the line (P = 1)
        if (d == 0) {
            line = b(j, 0) | b(j, 1) << 1 | b(k, 0) << 2 | b(j, 2) << 3 | b(k, 1) << 4 | b(k, 2) << 5;
            pos = i;
        } else if (d == 1) {
            line = b(i, 0) | b(i, 1) << 1 | b(k, 0) << 2 | b(i, 2) << 3 | b(k, 1) << 4 | b(k, 2) << 5;
            pos = j;
        } else {
            line = b(i, 0) | b(i, 1) << 1 | b(j, 1) << 2 | b(i, 2) << 3 | b(j, 0) << 4 | b(j, 2) << 5;
            pos = k;
        }
    } else if constexpr (NQ == 4) {   // two lines per row: row = line >> 1
        if (d == 0) {
            line = b(k, 1) | b(j, 0) << 1 | b(j, 1) << 2 | b(k, 0) << 3;
            pos = i;
        } else if (d == 1) {
            line = b(k, 1) | b(i, 0) << 1 | b(i, 1) << 2 | b(k, 0) << 3;
            pos = j;
        } else {
            line = b(j, 0) | b(i, 0) << 1 | b(i, 1) << 2 | b(j, 1) << 3;
            pos = k;
        }
    } else if (d == 0) {
        line = j + NQ * k;
        pos = i;
    } else if (d == 1) {
        line = i + NQ * k;
        pos = j;
    } else {
        line = i + NQ * j;
        pos = k;
    }
    const int lb = el * S::NL + line;
    return tc_slot(lb / S::P, (lb % S::P) * NQ + pos, S::LBO_A);
}

// Zeroes A and B and writes B1 = [Dh; Dl] and B2 = [Dh; 0] of this order.
template <int NQ>
__device__ void tc_prepare_operands(unsigned char *sm) {
    using S = TcShape<NQ>;
    uint4 *z = reinterpret_cast<uint4 *>(sm);
    for (int x = threadIdx.x; x < S::SMEM / 16; x += kThreads) z[x] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    float *B1 = reinterpret_cast<float *>(sm + 2 * S::REGION);
    float *B2 = reinterpret_cast<float *>(sm + 2 * S::REGION + S::BBYTES);
    const TcDiff &T = c_tc_diff[NQ];
    for (int x = threadIdx.x; x < S::NN * S::KW; x += kThreads) {
        const int row = x / S::KW, kk = x % S::KW;
        const bool tail = row >= S::H;
        const int r = tail ? row - S::H : row;
        if (r < S::PQ && kk < S::PQ && r / NQ == kk / NQ) {
            const int e = (r % NQ) * NQ + kk % NQ;
            const int o = tc_slot(row, kk, S::LBO_B) / 4;
            B1[o] = tail ? T.l[e] : T.h[e];
            B2[o] = tail ? 0.f : T.h[e];
        }
    }
}

// Writes the sums of K step ks of row R (heads' and tails' accumulator
// halves added) back into the row's flux slots; slots past the row's lines
// keep their zeros.
template <int NQ>
__device__ __forceinline__ void tc_store_row(unsigned char *Ah, int R, int ks, const uint32_t (&hv)[8],
                                             const uint32_t (&lv)[8]) {
    using S = TcShape<NQ>;
    unsigned char *row = Ah + (R >> 3) * 128 + (R & 7) * 16;
    float o[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) o[t] = __uint_as_float(hv[t]) + __uint_as_float(lv[t]);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int s0 = 8 * ks + 4 * c;   // first K slot of this chunk
        float *dst = reinterpret_cast<float *>(row + (2 * ks + c) * S::LBO_A);
        if (s0 + 3 < S::PQ) {
            *reinterpret_cast<float4 *>(dst) = make_float4(o[4 * c], o[4 * c + 1], o[4 * c + 2], o[4 * c + 3]);
        } else {
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (s0 + t < S::PQ) dst[t] = o[4 * c + t];
        }
    }
}

// One tile: elements [e0, e0 + count) of instance I through nsteps steps.
// Returns false if the wait for the tensor core ran out (the caller stops).
template <int NQ>
__device__ bool run_tile_tc(const BatchInstance &I, int64_t e0, int64_t count, const float *sco,
                            int nsteps, double dt, unsigned char *sm, uint32_t tmem,
                            uint64_t *bar, uint32_t &phase, int *s_nq) {
    using S = TcShape<NQ>;
    if (*s_nq != NQ) {   // uniform: written before the last barrier
        tc_prepare_operands<NQ>(sm);
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) *s_nq = NQ;
    }
    const int l = threadIdx.x, w = l >> 5, lane = l & 31;
    int el, i, j, k;
    tc_thread_point<NQ>(l, el, i, j, k);
    const int p = i + NQ * j + S::NL * k;
    const bool has_point = l < S::EPP * S::N3;
    unsigned char *Ah = sm;
    float *aux = reinterpret_cast<float *>(sm + kTcOperandBytes) + l;   // [word * kThreads]
    int *auxi = reinterpret_cast<int *>(aux);
#pragma unroll
    for (int d = 0; d < 3; ++d)
        auxi[(4 + d) * kThreads] = d * 5 * S::BLK_BYTES + tc_point_offset<NQ>(d, el, i, j, k);
    const uint32_t lane_base = tmem + ((uint32_t)(32 * (w & 3)) << 16);
    const uint32_t st_col = lane_base + kTcStateCol + kTcStateStride * (uint32_t)(w >> 2);
    const int64_t M = I.M;
    float *qv = static_cast<float *>(I.q);
    const float dtt = static_cast<float>(dt);
    const float grav = I.mp.grav;

    // passes in 32-bit counters (a work item holds far fewer than 2^31
    // elements); the point's global index is formed where it is used
    const int cnt = (int)count;
    for (int b0 = 0; b0 < cnt; b0 += S::EPP) {
        const int npass = cnt - b0 < S::EPP ? cnt - b0 : S::EPP;
        const bool active = has_point && el < npass;
        // v: q (0-4), g (5-13), J^-1 (14) of this thread's point.  It is kept
        // in registers from phase 3 into the next stage's phase 1, and
        // reloaded from TMEM for phase 3 (issued before the barrier that
        // precedes it, so the load's latency hides behind the barrier).
        uint32_t v[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) v[t] = 0u;
        if (active) {
            const int64_t node = (e0 + b0 + el) * S::N3 + p;
#pragma unroll
            for (int b = 0; b < kFields; ++b) v[b] = __float_as_uint(qv[b * M + node]);
#pragma unroll
            for (int s2 = 0; s2 < 9; ++s2) v[5 + s2] = __float_as_uint(__ldg(I.mgeo.g[s2] + node));
            v[14] = __float_as_uint(__ldg(I.mgeo.Jinv + node));
            const float th0 = __ldg(I.mgeo.theta_ref + node);
            EosRef32 er{0.f, 0.f};
            if (th0 > 0.f) er = eos_reference_f32(th0, I.mp);
            aux[0] = th0;
            aux[kThreads] = __ldg(I.mgeo.rho_ref + node);
            aux[2 * kThreads] = er.w;
            aux[3 * kThreads] = er.A;
        }
        {
            uint32_t z[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            tc::tmem_st16(st_col, v);
            tc::tmem_st8(st_col + 16, z);
        }

        for (int step = 0; step < nsteps; ++step) {
#pragma unroll 1
            for (int st = 0; st < 5; ++st) {
                // Phase 3 reads and phase 1 writes only the thread's own
                // point's slots of A (the stage's MMAs completed before the
                // readback); the first stage of a pass takes a barrier, since
                // the previous pass or work item gave its slots to other threads.
                if (step == 0 && st == 0) __syncthreads();
                // ---- phase 1: p', fluxes, heads and tails into A -------
                if (active) {
                    const float th0 = aux[0], rho0 = aux[kThreads];
                    const EosRef32 er{aux[2 * kThreads], aux[3 * kThreads]};
                    float q[kFields], g[9];
#pragma unroll
                    for (int b = 0; b < kFields; ++b) q[b] = __uint_as_float(v[b]);
#pragma unroll
                    for (int s2 = 0; s2 < 9; ++s2) g[s2] = __uint_as_float(v[5 + s2]);
                    const float rho = rho0 + q[0];
                    const float Th = th0 + q[4];
                    const float pp = pressure_perturbation_f32(q[4], th0, er, I.mp);
                    const float rinv = __frcp_rn(rho);   // the correctly rounded 1/rho
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const float g1 = g[3 * d], g2 = g[3 * d + 1], g3 = g[3 * d + 2];
                        const float vv = fmaf(g3, q[3], fmaf(g2, q[2], g1 * q[1]));
                        const float u = vv * rinv;
                        const float F[kFields] = {vv, fmaf(q[1], u, g1 * pp), fmaf(q[2], u, g2 * pp),
                                                  fmaf(q[3], u, g3 * pp), Th * u};
                        unsigned char *ad = Ah + auxi[(4 + d) * kThreads];
#pragma unroll
                        for (int b = 0; b < kFields; ++b) {
                            unsigned char *a = ad + b * S::BLK_BYTES;
                            *reinterpret_cast<float *>(a) = F[b];
                            *reinterpret_cast<float *>(a + S::REGION) = F[b] - tf32_head_dev(F[b]);
                        }
                    }
                }
                tc::fence_proxy_async_smem();
                tc::fence_before_sync();
                __syncthreads();
                // ---- phase 2: the split products on the tensor core ----
                if (l == 0) {
                    tc::fence_after_sync();
                    constexpr uint32_t idesc = tc::idesc_tf32(128, S::NN);
                    const uint32_t ah = smem_addr(sm), al = ah + S::REGION;
                    const uint32_t b1 = ah + 2 * S::REGION, b2 = b1 + S::BBYTES;
#pragma unroll 1
                    for (int m = 0; m < S::NBLK; ++m) {
#pragma unroll
                        for (int ks = 0; ks < S::KS; ++ks) {
                            const uint32_t ao = m * 2048 + 2 * ks * S::LBO_A, bo = 2 * ks * S::LBO_B;
                            tc::mma_tf32(tmem + m * S::NN, tc::smem_desc(ah + ao, S::LBO_A, 128),
                                         tc::smem_desc(b1 + bo, S::LBO_B, 128), idesc, ks > 0);
                            tc::mma_tf32(tmem + m * S::NN, tc::smem_desc(al + ao, S::LBO_A, 128),
                                         tc::smem_desc(b2 + bo, S::LBO_B, 128), idesc, 1);
                        }
                    }
                    tc::mma_commit(bar);
                }
                const bool ok = bulk_wait(bar, phase);
                if (__syncthreads_or(!ok)) return false;
                phase ^= 1u;
                tc::fence_after_sync();
                // ---- readback: C[:, 0:H] + C[:, H:2H] into the flux slots ----
                // A warp reads the blocks m = warp / 4 + 4 t of its lane quarter.
                // (Issuing a warp's loads of two blocks before one wait needs
                // 32 more live registers and spills at this kernel's 64.)
#pragma unroll 1
                for (int m = w >> 2; m < S::NBLK; m += 4) {
                    const int R = m * 128 + 32 * (w & 3) + lane;
#pragma unroll
                    for (int ks = 0; ks < S::KS; ++ks) {
                        uint32_t hv[8], lv[8];
                        tc::tmem_ld8(lane_base + m * S::NN + 8 * ks, hv);
                        tc::tmem_ld8(lane_base + m * S::NN + S::H + 8 * ks, lv);
                        tc::tmem_ld_wait8x2(hv, lv);
                        tc_store_row<NQ>(Ah, R, ks, hv, lv);
                    }
                }
                // the state for phase 3 (its stores of the last stage are complete first)
                uint32_t dv[8];
                tc::tmem_st_wait();
                tc::tmem_ld16(st_col, v);
                tc::tmem_ld8(st_col + 16, dv);
                tc::fence_before_sync();
                __syncthreads();
                // ---- phase 3: rhs, stage update ------------------------
                tc::tmem_ld_wait16(v);
                tc::tmem_ld_wait(dv);
                if (active) {
                    const float a = sco[st], bcoef = sco[5 + st];
                    const float jinv = __uint_as_float(v[14]);
                    const float drho = __uint_as_float(v[0]);   // rho - rho_ref before the update
                    const unsigned char *a0 = Ah + auxi[4 * kThreads], *a1 = Ah + auxi[5 * kThreads],
                                        *a2 = Ah + auxi[6 * kThreads];
#pragma unroll
                    for (int b = 0; b < kFields; ++b) {
                        const float Rb = *reinterpret_cast<const float *>(a0 + b * S::BLK_BYTES) +
                                         *reinterpret_cast<const float *>(a1 + b * S::BLK_BYTES) +
                                         *reinterpret_cast<const float *>(a2 + b * S::BLK_BYTES);
                        float rhs = -jinv * Rb;
                        if (b == 3) rhs = fmaf(-drho, grav, rhs);
                        const float dq = fmaf(a, __uint_as_float(dv[b]), dtt * rhs);
                        dv[b] = __float_as_uint(dq);
                        v[b] = __float_as_uint(fmaf(bcoef, dq, __uint_as_float(v[b])));
                    }
                }
                {
                    uint32_t q8[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) q8[t] = v[t];
                    tc::tmem_st8(st_col, q8);
                    tc::tmem_st8(st_col + 16, dv);
                }
            }
        }
        tc::tmem_st_wait();
        if (active) {
            const int64_t node = (e0 + b0 + el) * S::N3 + p;
            float *q_out = static_cast<float *>(I.q);
            const int64_t Mo = I.M;
#pragma unroll
            for (int b = 0; b < kFields; ++b) q_out[b * Mo + node] = __uint_as_float(v[b]);
        }
    }
    return true;
}

// The CUDA-core tile (run_tile's phases: fluxes by point into the line
// layout of element_sweep.cuh, even-odd sweeps by line, combination by point)
// with each point's q, dq, metric terms and J^-1 in tensor memory (the columns
// run_tile_tc uses) instead of shared memory: shared memory holds only the
// fluxes, and the point phases read and write the state with three TMEM
// loads and two TMEM stores per stage instead of 35 shared accesses.
template <int NQ>
__device__ void run_tile_cc_tm(const BatchInstance &I, int64_t e0, int64_t count, const float *sco,
                               int nsteps, double dt, unsigned char *sm, uint32_t tmem) {
    constexpr int N3 = NQ * NQ * NQ;
    constexpr int NL = NQ * NQ;
    constexpr int EPP = kThreads / N3;
    constexpr int EW = block_words<NQ, float>();
    constexpr int BLK = EPP * EW;
    constexpr int TASKS = 3 * kFields * EPP * NL;
    float *sF = reinterpret_cast<float *>(sm);
    float *aux = reinterpret_cast<float *>(sm + kTcOperandBytes) + threadIdx.x;
    const int l = threadIdx.x, w = l >> 5;
    const int el = l / N3, p = l % N3;
    const int i = p % NQ, j = (p / NQ) % NQ, k = p / NL;
    const bool has_point = l < EPP * N3;
    int f[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) f[d] = d * kFields * BLK + el * EW + dir_slot<NQ, float>(d, i, j, k);
    const uint32_t st_col =
        tmem + ((uint32_t)(32 * (w & 3)) << 16) + kTcStateCol + kTcStateStride * (uint32_t)(w >> 2);
    const float dtt = static_cast<float>(dt);
    const float grav = I.mp.grav;
    const int cnt = (int)count;
    for (int b0 = 0; b0 < cnt; b0 += EPP) {
        const int npass = cnt - b0 < EPP ? cnt - b0 : EPP;
        const bool active = has_point && el < npass;
        uint32_t v[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) v[t] = 0u;
        if (active) {
            const int64_t node = (e0 + b0 + el) * N3 + p;
            const float *qv = static_cast<const float *>(I.q);
#pragma unroll
            for (int b = 0; b < kFields; ++b) v[b] = __float_as_uint(qv[b * I.M + node]);
#pragma unroll
            for (int s2 = 0; s2 < 9; ++s2) v[5 + s2] = __float_as_uint(__ldg(I.mgeo.g[s2] + node));
            v[14] = __float_as_uint(__ldg(I.mgeo.Jinv + node));
            const float th0 = __ldg(I.mgeo.theta_ref + node);
            EosRef32 er{0.f, 0.f};
            if (th0 > 0.f) er = eos_reference_f32(th0, I.mp);
            aux[0] = th0;
            aux[kThreads] = __ldg(I.mgeo.rho_ref + node);
            aux[2 * kThreads] = er.w;
            aux[3 * kThreads] = er.A;
        }
        {
            uint32_t z[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            tc::tmem_st16(st_col, v);
            tc::tmem_st8(st_col + 16, z);
        }
        for (int step = 0; step < nsteps; ++step) {
#pragma unroll 1
            for (int st = 0; st < 5; ++st) {
                // Phase 3 reads and phase 1 writes only the thread's own
                // point's flux slots, so within a pass the next stage's phase 1
                // needs no barrier after phase 3.  The first stage of a pass
                // takes one: the previous pass or work item (possibly another
                // order) gave its slots to other threads.
                if (step == 0 && st == 0) __syncthreads();
                if (active) {
                    const float th0 = aux[0], rho0 = aux[kThreads];
                    const EosRef32 er{aux[2 * kThreads], aux[3 * kThreads]};
                    float q[kFields], g[9];
#pragma unroll
                    for (int b = 0; b < kFields; ++b) q[b] = __uint_as_float(v[b]);
#pragma unroll
                    for (int s2 = 0; s2 < 9; ++s2) g[s2] = __uint_as_float(v[5 + s2]);
                    const float rho = rho0 + q[0];
                    const float Th = th0 + q[4];
                    const float pp = pressure_perturbation_f32(q[4], th0, er, I.mp);
                    const float rinv = __frcp_rn(rho);   // the correctly rounded 1/rho
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const float g1 = g[3 * d], g2 = g[3 * d + 1], g3 = g[3 * d + 2];
                        const float vv = fmaf(g3, q[3], fmaf(g2, q[2], g1 * q[1]));
                        const float u = vv * rinv;
                        float *F = sF + f[d];
                        F[0 * BLK] = vv;
                        F[1 * BLK] = fmaf(q[1], u, g1 * pp);
                        F[2 * BLK] = fmaf(q[2], u, g2 * pp);
                        F[3 * BLK] = fmaf(q[3], u, g3 * pp);
                        F[4 * BLK] = Th * u;
                    }
                }
                __syncthreads();
#pragma unroll 1
                for (int t = l; t < TASKS; t += kThreads) {
                    const int bd = t / (EPP * NL), rem = t % (EPP * NL);
                    const int e = rem / NL, line = rem % NL;
                    if (e < npass) sweep_line<NQ>(sF + bd * BLK + e * EW, line, c_sweep32[NQ]);
                }
                // the state for phase 3, its loads issued before the barrier
                uint32_t dv[8];
                tc::tmem_st_wait();
                tc::tmem_ld16(st_col, v);
                tc::tmem_ld8(st_col + 16, dv);
                __syncthreads();
                tc::tmem_ld_wait16(v);
                tc::tmem_ld_wait(dv);
                if (active) {
                    const float a = sco[st], bcoef = sco[5 + st];
                    const float jinv = __uint_as_float(v[14]);
                    const float drho = __uint_as_float(v[0]);
#pragma unroll
                    for (int b = 0; b < kFields; ++b) {
                        const float R = sF[f[0] + b * BLK] + sF[f[1] + b * BLK] + sF[f[2] + b * BLK];
                        float rhs = -jinv * R;
                        if (b == 3) rhs = fmaf(-drho, grav, rhs);
                        const float dq = fmaf(a, __uint_as_float(dv[b]), dtt * rhs);
                        dv[b] = __float_as_uint(dq);
                        v[b] = __float_as_uint(fmaf(bcoef, dq, __uint_as_float(v[b])));
                    }
                }
                {
                    uint32_t q8[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) q8[t] = v[t];
                    tc::tmem_st8(st_col, q8);
                    tc::tmem_st8(st_col + 16, dv);
                }
            }
        }
        tc::tmem_st_wait();
        if (active) {
            const int64_t node = (e0 + b0 + el) * N3 + p;
            float *q_out = static_cast<float *>(I.q);
#pragma unroll
            for (int b = 0; b < kFields; ++b) q_out[b * I.M + node] = __uint_as_float(v[b]);
        }
    }
}

}  // namespace

}  // namespace numa
