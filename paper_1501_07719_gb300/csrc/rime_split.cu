// rime_split.cu -- the RIME predict / chi^2 of point sources on the tcgen05
// tensor cores, in split precision.
//
// With point sources the per-baseline source sum factors through the
// per-antenna terms A_tpsk = E_tpsk K_tpsk (eqs. 3-4): for each (t, k) and
// each Stokes parameter X in (I, Q, U, V),
//
//   S_X[p, q] = sum_s A_ps X_s conj(A_qs)  =  (A diag(X) A^H)[p, q],
//
// a complex matrix product over the sources (the sum of Algorithm 2 for all
// baselines at once). With the source index and the real/imaginary part as
// the contraction index (K = 2 nsrc) it is two real products,
//
//   Re S_X[p, q] = sum_s [Re A_ps, Im A_ps] . X_s [Re A_qs, Im A_qs]
//   Im S_X[p, q] = sum_s [Re A_ps, Im A_ps] . X_s [-Im A_qs, Re A_qs],
//
// which the tensor cores evaluate in FP32 from operands split into a high
// and a low part (x = hi + lo, hi = x rounded to BF16 or TF32, lo = the
// rounded remainder): x y ~ hi_x hi_y + hi_x lo_y + lo_x hi_y, three MMAs
// per product; the lo_x lo_y term (relative 2^-16 for BF16, 2^-22 for TF32)
// is dropped.
//
// One CTA owns (t, k) and a tile of 128 row antennas p (the MMA's M, one
// TMEM lane each: four groups of 32 antennas, see split_tiles) by a group of
// 32 column antennas q; the B operand has one row per
// (q, X) for the real parts and one per (q, X) for the imaginary parts,
// N = 256, so one MMA reads A once for both. Twelve producer warps form the
// operands of each chunk of
// sources straight into shared memory: the phase nu tau is reduced exactly in
// double-float arithmetic (the delays tau come from the FP64 upload kernel)
// and its sine and cosine are taken with the SFU; one thread issues the
// MMAs; an eight-stage mbarrier pipeline connects them.
//
// The tensor core adds each MMA's products into its FP32 accumulator with
// truncation, losing about one unit in the last place of the running sum per
// MMA, a bias toward zero that grows with the number of MMAs into one
// accumulator. So the accumulators (Re and Im, 128 columns each) live in two
// TMEM buffers used in turn for segments of eight stages: while the MMAs fill
// one, the A producer warps add the other into FP32 running sums held in
// their registers (round to nearest; the warpgroups' register budgets are
// rebalanced with setmaxnreg so that each A thread can hold its 128 sums).
// The epilogue applies the Stokes combination
// (eq. 2) and the gains (eq. 1) to the running sums and writes V or forms
// w |V - D|^2 (eq. 7), summed in FP64.
#include "rime_internal.cuh"
#include "rime_dev.cuh"
#include "rime_tc.cuh"
#include "rime_beam.cuh"
#include "rime_fused_common.cuh"

#include <algorithm>
#include <vector>

namespace rime {
namespace split {

constexpr int PT = 128;                 // row antennas per tile (MMA M)
constexpr int QT = 32;                  // column antennas per tile
constexpr int NB = 8 * QT;              // B rows: (q, X) for Re S, then i (q, X) for Im S; MMA N
constexpr int NDRAIN = 256;             // A producers, which also drain and run the epilogue
constexpr int NPROD = NDRAIN + 128;     // and four warps of B producers
constexpr int THREADS = NPROD + 128;    // and a warpgroup whose first warp issues the MMAs
constexpr int NST = 8;                  // pipeline stages
// registers per thread: at launch (65536 / THREADS), then per warpgroup
// A (two warpgroups: 128 running sums each), B, MMA, e.g. 2*128*200 +
// 128*88 + 128*24 = 65536 = 128 * 512
// (BF16: 208 for A, 72 for B; TF32, whose B threads need more: 200 and 88)
#ifndef RIME_SPLIT_REGS_A_BF16
#define RIME_SPLIT_REGS_A_BF16 208
#endif
#ifndef RIME_SPLIT_REGS_A_TF32
#define RIME_SPLIT_REGS_A_TF32 200
#endif
constexpr int REGS_LAUNCH = 128, REGS_MMA = 24;
template <bool TF32> struct Regs {
    static constexpr int A = TF32 ? RIME_SPLIT_REGS_A_TF32 : RIME_SPLIT_REGS_A_BF16;
    static constexpr int B = (REGS_LAUNCH * THREADS - 2 * 128 * A - 128 * REGS_MMA) / 128 / 8 * 8;
    static_assert(2 * 128 * A + 128 * B + 128 * REGS_MMA <= REGS_LAUNCH * THREADS, "register split");
    static_assert(A % 8 == 0 && A <= 256 && B >= 24 && B <= REGS_LAUNCH, "setmaxnreg range");
};
constexpr int SEG = 8;                  // stages accumulated in TMEM before a drain
constexpr uint32_t A_BYTES = tc::operand_bytes(PT);
constexpr uint32_t B_BYTES = tc::operand_bytes(NB);
// one stage: A hi, A lo, B hi, B lo
constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr uint32_t SMEM_BYTES = NST * STAGE_BYTES;
constexpr uint32_t TMEM_COLS = 512;     // two buffers of (Re, Im) x 128 columns
static_assert(SMEM_BYTES + 1024 <= 227 * 1024, "shared memory");
// the epilogue stores the running sums ([256 columns][128 rows] of float)
// in the stage buffers, so they must hold them
static_assert(SMEM_BYTES >= 256u * 128u * 4u, "stage buffers smaller than the epilogue's sums");
static_assert(STAGE_BYTES % 16 == 0 && A_BYTES % 16 == 0 && B_BYTES % 16 == 0, "operand alignment");

struct SplitParams {
    int na, ntime, nchan, nsrc, ntiles;
    long long nbl;
    int has_gains, has_weight, has_pointing;
    const int2 *tiles;        // (column group, packed row groups) of each tile (split_tiles)
    const ChanF *chan;
    const float2 *tau;        // [ntime][nsrc][na] double-float delays (s)
    const float *rho;         // [ntime][nsrc][na] beam radii
    const float *scale;       // [scale_trows][nchan][nsrc][4]: X_s (nu/nu_ref)^alpha, times E_s^2 without pointing
    int scale_trows;          // ntime (time-varying brightness) or 1
    int nsrc_pad;             // sources per scale row: nsrc rounded up to a whole stage, zero past nsrc
    const float2 *gains;      // [ntime][na][nchan][4]
    const float2 *data;       // [ntime][nbl][nchan][4]
    const float *weight;      // [ntime][nbl][nchan]
    float2 *vis_out;
    double *partials;
    unsigned *counter;
    double *result;
    DevStatus *status;
    unsigned long long wait_ns;   // limit of the bounded waits
};

// K = exp(2 pi i nu tau) with nu tau reduced exactly to about [-1/2, 1/2]
// turns in double-float arithmetic, then the SFU sine and cosine (the same
// routine as the direct FP32 kernels).
__device__ __forceinline__ float2 phase_sfu(float2 tau, const ChanF &ch) { return f32::phase_factor(tau, ch); }
__device__ __forceinline__ float beam_f(float rho, const ChanF &ch) { return beam_E(ch.beam, ch.cnu * rho); }

// (x, y) -> packed hi and lo words: BF16 pairs (x in the low half).
__device__ __forceinline__ uint32_t pack_bf16(float x, float y) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(y), "f"(x));
    return r;
}
// x = hi + lo with hi = x rounded to nearest BF16 and lo = x - hi, which is
// exact in FP32 (the error of rounding to 8 significant bits needs at most
// 16), then rounded to BF16. hi is unpacked from its word by shifts.
__device__ __forceinline__ void split_bf16(float x, float y, uint32_t &hi, uint32_t &lo) {
    hi = pack_bf16(x, y);
    const float xh = __uint_as_float(hi << 16), yh = __uint_as_float(hi & 0xffff0000u);
    lo = pack_bf16(__fsub_rn(x, xh), __fsub_rn(y, yh));
}
// split_bf16 and the split words of i (x + i y) = -y + i x, converted
// directly (rounding commutes with negation).
__device__ __forceinline__ void split_bf16_rot(float x, float y, uint32_t &hi, uint32_t &lo, uint32_t &hr,
                                               uint32_t &lr) {
    hi = pack_bf16(x, y);
    hr = pack_bf16(-y, x);
    const float dx = __fsub_rn(x, __uint_as_float(hi << 16)), dy = __fsub_rn(y, __uint_as_float(hi & 0xffff0000u));
    lo = pack_bf16(dx, dy);
    lr = pack_bf16(-dy, dx);
}
// FP16 pairs: the same split as BF16 with the FP16 rounding (11 significant
// bits, as TF32, and the 16-bit operands of BF16); hi is unpacked by
// conversion. A remainder below 2^-14 is an FP16 subnormal (absolute
// spacing 2^-24): a value of magnitude below 1/8 then keeps an absolute error
// of at most 2^-25 instead of a relative one, which the sums, scaled by
// |A| <= 1 or the source's flux, tolerate.
__device__ __forceinline__ uint32_t pack_f16(float x, float y) {
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(y), "f"(x));
    return r;
}
__device__ __forceinline__ void unpack_f16(uint32_t w, float &x, float &y) {
    asm("{\n\t.reg .f16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;\n\t}"
        : "=f"(x), "=f"(y)
        : "r"(w));
}
__device__ __forceinline__ void split_f16(float x, float y, uint32_t &hi, uint32_t &lo) {
    hi = pack_f16(x, y);
    float xh, yh;
    unpack_f16(hi, xh, yh);
    lo = pack_f16(__fsub_rn(x, xh), __fsub_rn(y, yh));
}
__device__ __forceinline__ void split_f16_rot(float x, float y, uint32_t &hi, uint32_t &lo, uint32_t &hr,
                                              uint32_t &lr) {
    hi = pack_f16(x, y);
    hr = pack_f16(-y, x);
    float xh, yh;
    unpack_f16(hi, xh, yh);
    const float dx = __fsub_rn(x, xh), dy = __fsub_rn(y, yh);
    lo = pack_f16(dx, dy);
    lr = pack_f16(-dy, dx);
}
// Operand formats of the split modes.
enum : int { FMT_BF16 = 0, FMT_TF32 = 1, FMT_F16 = 2 };

// TF32: round to nearest (ties away) into the 19 bits the tensor core reads.
__device__ __forceinline__ uint32_t tf32_bits(float x) { return (__float_as_uint(x) + 0x1000u) & 0xffffe000u; }
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    hi = tf32_bits(x);
    lo = tf32_bits(x - __uint_as_float(hi));
}

__device__ __forceinline__ void st16(unsigned char *p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    *reinterpret_cast<uint4 *>(p) = make_uint4(a, b, c, d);
}

// Operands of one pipeline stage: BF16 8 sources (K = 16), TF32 4 (K = 8),
// as two 16-byte chunks per operand row. Element (row, source j, part c)
// sits at K index 2 j + c. Warps 0-7 form A (thread: row p, chunk), drain
// the accumulators and run the epilogue; warps 8-11 form B (thread: antenna
// q, chunk and a pair of Stokes parameters: rows (q, X) and i (q, X) from one
// phase); warp 12 issues the MMAs; warps 13-15 only lend their registers. Sources past the end read the last source's delays and
// meet a zero Stokes scale, so they add nothing; rows and columns past the
// last antenna are never read back.
template <bool TF32>
struct Item {
    static constexpr int SPC = TF32 ? 2 : 4;   // sources per chunk
    static constexpr int SPS = 2 * SPC;        // sources per stage
};

// State shared by the roles of one CTA.
struct Cta {
    const SplitParams &P;
    unsigned char *smem;
    uint64_t *full, *empty, *seg_full, *seg_empty, *drained;
    int *abort_flag;
    uint32_t tmem;
    int t, k, cg, nstg, nseg;
    uint32_t rows;   // row groups of the tile: 8 bits per 32-row slot, 0xff empty
    ChanF ch;
};

// Inputs of one chunk of one producer thread, loaded a stage ahead (beam
// radii, needed only with pointing errors, are loaded where used).
template <int SPC>
struct Pre {
    float2 tau[SPC];
    float2 x[SPC];   // B: the Stokes pair (X = 2 xp, 2 xp + 1) of each source
};

// Waits for pipeline slot `it` to be free; A warps drain finished segments
// meanwhile. Warp-uniform; false when the block gave up.
template <typename Drain>
__device__ __forceinline__ bool wait_slot(const Cta &C, int it, int lane, Drain &&maybe_drain) {
    const int slot = it % NST;
    const uint32_t par = ((it / NST) & 1) ^ 1;
    const uint64_t t0 = tc::global_ns();
    for (uint32_t i = 0;; i++) {
        // a completed phase stays complete until this slot is refilled, so
        // the lanes agree once all have seen it
        if (__all_sync(0xffffffffu, tc::mbar_try_wait_sleep(&C.empty[slot], par, 1000u))) return true;
        maybe_drain();
        const bool check = C.P.wait_ns < 1000000ull || (i & 63) == 63;
        if (check &&
            __any_sync(0xffffffffu, *(volatile int *)C.abort_flag != 0 || tc::global_ns() - t0 > C.P.wait_ns))
            return false;
    }
}

// Warps 0-7: A = E K rows (row p, chunk), the drains into register sums, and
// the epilogue. Returns this thread's chi^2 contribution.
template <int FMT, bool WRITE>
__device__ __forceinline__ double role_a(const Cta &C, int tid, int warp, int lane) {
    constexpr bool TF32 = FMT == FMT_TF32;
    constexpr int SPC = Item<TF32>::SPC, SPS = Item<TF32>::SPS;
    const SplitParams &P = C.P;
    const int row = tid & 127, chunk = tid >> 7;
    const int rgrp = (C.rows >> (8 * (row >> 5))) & 0xff;   // 0xff: an empty slot, formed from antenna 0
    const int ant = rgrp == 0xff ? 0 : min(QT * rgrp + (row & 31), P.na - 1);
    const long long tbase = (long long)C.t * P.nsrc * P.na + ant;
    const uint32_t o_row = tc::operand_offset(row, 16 * chunk);
    const bool pointing = P.has_pointing != 0;
    const int quad = warp & 3, half = (warp >> 2) & 1;
    const int lrow = 32 * quad + lane;
    const ChanF ch = C.ch;

    const float2 *tau0 = P.tau + tbase;
    const int na = P.na, last = P.nsrc - 1;
    auto load = [&](int it, Pre<SPC> &L) {
        const int sb = it * SPS + chunk * SPC;
        if (sb + SPC - 1 <= last) {   // all sources live (warp-uniform)
            const float2 *p = tau0 + (size_t)sb * na;
#pragma unroll
            for (int j = 0; j < SPC; j++) L.tau[j] = p[j * na];
        } else {
#pragma unroll
            for (int j = 0; j < SPC; j++) L.tau[j] = tau0[(size_t)min(sb + j, last) * na];
        }
    };
    // FP32 running sums of this thread's accumulator columns: Re S then Im S
    // for columns 64 half .. 64 half + 63 of each
    float tot[128];
#pragma unroll
    for (int c = 0; c < 128; c++) tot[c] = 0.f;
    int nd = 0;   // next segment to drain
    auto drain = [&]() {
        const int b = nd & 1;
        tc::tc_fence_after();
#pragma unroll
        for (int h = 0; h < 2; h++)   // Re, Im
#pragma unroll
            for (int c4 = 0; c4 < 4; c4++) {
                uint32_t r[16];
                const int col0 = 128 * h + 64 * half + 16 * c4;
                tc::tmem_ld16(C.tmem + ((uint32_t)(32 * quad) << 16) + 256 * b + col0, r);
                tc::tmem_wait_ld16(r);
#pragma unroll
                for (int c = 0; c < 16; c++) tot[64 * h + 16 * c4 + c] += __uint_as_float(r[c]);
            }
        tc::tc_fence_before();
        tc::mbar_arrive(&C.seg_empty[b]);
        nd++;
    };
    // warp-uniform: drain the next segment if it is complete
    auto maybe_drain = [&]() {
        bool r = false;
        if (lane == 0) r = nd < C.nseg && tc::mbar_try_wait(&C.seg_full[nd & 1], (nd >> 1) & 1);
        if (__shfl_sync(0xffffffffu, r, 0)) drain();
    };
    auto produce = [&](int it, const Pre<SPC> &L) {
        unsigned char *stg = C.smem + (it % NST) * STAGE_BYTES;
        float2 a[SPC];
#pragma unroll
        for (int j = 0; j < SPC; j++) {
            a[j] = phase_sfu(L.tau[j], ch);
            if (pointing) {
                const int s = min(it * SPS + chunk * SPC + j, P.nsrc - 1);
                const float E = beam_f(P.rho[tbase + (long long)s * P.na], ch);
                a[j].x *= E;
                a[j].y *= E;
            }
        }
        uint32_t h[4], l[4];
        if (TF32) {
#pragma unroll
            for (int j = 0; j < SPC; j++) {
                split_tf32(a[j].x, h[2 * j], l[2 * j]);
                split_tf32(a[j].y, h[2 * j + 1], l[2 * j + 1]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < SPC; j++) {
                if (FMT == FMT_F16) split_f16(a[j].x, a[j].y, h[j], l[j]);
                else split_bf16(a[j].x, a[j].y, h[j], l[j]);
            }
        }
        st16(stg + o_row, h[0], h[1], h[2], h[3]);
        st16(stg + A_BYTES + o_row, l[0], l[1], l[2], l[3]);
    };
    // Two stages per proxy fence and pair of arrivals (a fixed cost per stage;
    // on a 256-antenna slice BF16 -3.5 %, TF32 -9 % with the B warps paired
    // too); each stage's delays are loaded two stages ahead.
    Pre<SPC> b0, b1;
    if (C.nstg > 0) load(0, b0);
    if (C.nstg > 1) load(1, b1);
    bool ok = true;
    for (int it = 0; it < C.nstg && ok; it += 2) {
        const bool two = it + 1 < C.nstg;
        ok = wait_slot(C, it, lane, maybe_drain);
        if (!ok) break;
        produce(it, b0);
        if (it + 2 < C.nstg) load(it + 2, b0);
        if (two) {
            ok = wait_slot(C, it + 1, lane, maybe_drain);
            if (!ok) break;
            produce(it + 1, b1);
            if (it + 3 < C.nstg) load(it + 3, b1);
        }
        tc::fence_async_smem();
        tc::mbar_arrive(&C.full[it % NST]);
        if (two) tc::mbar_arrive(&C.full[(it + 1) % NST]);
        // a segment can only have finished once its last stage was formed
        if (it + 1 >= (nd + 1) * SEG) maybe_drain();
    }
    while (ok && nd < C.nseg) {   // the remaining segments
        const bool got = __all_sync(0xffffffffu, tc::mbar_wait(&C.seg_full[nd & 1], (nd >> 1) & 1, C.abort_flag, P.wait_ns));
        if (!got) ok = false;
        else drain();
    }
    if (!ok) *(volatile int *)C.abort_flag = 1;
    ok = __all_sync(0xffffffffu, ok && *(volatile int *)C.abort_flag == 0);
    if (!ok) {
        if (lane == 0) atomicOr(&P.status->err[EC_RUN], EB_TIMEOUT);
        return 0.0;
    }

    // ---- epilogue: row lrow (antenna p) against columns q = 16 half .. 16 half + 15 of the column group ----
    // Every MMA has completed and every stage has been consumed, so the stage
    // buffers take this thread's sums ([256 columns][128 rows]); each thread
    // reads back only what it wrote.
    float *ts = reinterpret_cast<float *>(C.smem);
#pragma unroll
    for (int c = 0; c < 64; c++) {
        ts[(64 * half + c) * 128 + lrow] = tot[c];
        ts[(128 + 64 * half + c) * 128 + lrow] = tot[64 + c];
    }
    double chi = 0.0;
    const int rg = (C.rows >> (8 * quad)) & 0xff;   // the row group of slot quad
    const int pgl = QT * rg + lane;
    const bool prow = rg != 0xff && pgl < P.na;
    const bool same = rg == C.cg;   // pairs inside one group: p < q only
    const bool swap = rg > C.cg;    // p > q for the whole slot: the tile holds S_X[p, q] = conj S_X[q, p]
    const int t = C.t, k = C.k;
    float2 gp[4] = {{1.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {1.f, 0.f}};
    if (P.has_gains && prow) {
        const float4 *g4 = reinterpret_cast<const float4 *>(P.gains + 4 * (((long long)t * P.na + pgl) * P.nchan + k));
        const float4 a01 = g4[0], a23 = g4[1];
        gp[0] = make_float2(a01.x, a01.y); gp[1] = make_float2(a01.z, a01.w);
        gp[2] = make_float2(a23.x, a23.y); gp[3] = make_float2(a23.z, a23.w);
    }
    // two baselines per iteration: the second one's loads are issued before
    // the first one's arithmetic (BF16 -2 %, TF32 -1 % on a 256-antenna slice;
    // four or sixteen per iteration spill)
#pragma unroll 2
    for (int i = 0; i < 16; i++) {
        const int q = QT * C.cg + 16 * half + i;
        if (!(prow && q < P.na && (!same || pgl < q))) continue;
        float Sv[8];   // Re I, Q, U, V then Im I, Q, U, V
#pragma unroll
        for (int x = 0; x < 4; x++) {
            Sv[x] = ts[(64 * half + 4 * i + x) * 128 + lrow];
            Sv[4 + x] = ts[(128 + 64 * half + 4 * i + x) * 128 + lrow];
            if (swap) Sv[4 + x] = -Sv[4 + x];   // baseline (q, p): S_X[q, p]
        }
        float2 Sm[4];
        Sm[0] = make_float2(Sv[0] + Sv[1], Sv[4] + Sv[5]);   // I + Q
        Sm[1] = make_float2(Sv[2] - Sv[7], Sv[6] + Sv[3]);   // U + iV
        Sm[2] = make_float2(Sv[2] + Sv[7], Sv[6] - Sv[3]);   // U - iV
        Sm[3] = make_float2(Sv[0] - Sv[1], Sv[4] - Sv[5]);   // I - Q
        float2 gq[4] = {{1.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {1.f, 0.f}};
        if (P.has_gains) {
            const float4 *g4 = reinterpret_cast<const float4 *>(P.gains + 4 * (((long long)t * P.na + q) * P.nchan + k));
            const float4 b01 = g4[0], b23 = g4[1];
            gq[0] = make_float2(b01.x, b01.y); gq[1] = make_float2(b01.z, b01.w);
            gq[2] = make_float2(b23.x, b23.y); gq[3] = make_float2(b23.z, b23.w);
        }
        float2 V[4], tmp[4], gbh[4];
        // eq. 1 for the baseline (a, b), a < b: V = G_a S G_b^H
        mmul(swap ? gq : gp, Sm, tmp);
        mherm(swap ? gp : gq, gbh);
        mmul(tmp, gbh, V);
        const long long a = swap ? q : pgl, b = swap ? pgl : q;
        const long long vrow = ((long long)t * P.nbl + a * P.na - a * (a + 1) / 2 - a - 1 + b) * P.nchan + k;
        if (WRITE) {
            float4 *o = reinterpret_cast<float4 *>(P.vis_out + 4 * vrow);
            o[0] = make_float4(V[0].x, V[0].y, V[1].x, V[1].y);
            o[1] = make_float4(V[2].x, V[2].y, V[3].x, V[3].y);
        } else {
            const float4 *d4 = reinterpret_cast<const float4 *>(P.data + 4 * vrow);
            const float4 d01 = d4[0], d23 = d4[1];
            const float2 D[4] = {make_float2(d01.x, d01.y), make_float2(d01.z, d01.w),
                                 make_float2(d23.x, d23.y), make_float2(d23.z, d23.w)};
            float r2 = 0.f;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const float dr = V[c].x - D[c].x, di = V[c].y - D[c].y;
                r2 += dr * dr + di * di;
            }
            const float w = P.has_weight ? P.weight[vrow] : 1.f;
            chi += (double)(w * r2);
        }
    }
    return chi;
}

// Warps 8-11: B rows (antenna q, chunk, Stokes pair xp): X A_q and i X A_q
// for X = 2 xp, 2 xp + 1, from one phase per (q, source).
template <int FMT>
__device__ __forceinline__ void role_b(const Cta &C, int warp, int lane) {
    constexpr bool TF32 = FMT == FMT_TF32;
    constexpr int SPC = Item<TF32>::SPC, SPS = Item<TF32>::SPS;
    const SplitParams &P = C.P;
    const int bw = warp - NDRAIN / 32;
    const int chunk = bw & 1, xp = bw >> 1;
    const int row = lane;
    const int ant = min(QT * C.cg + row, P.na - 1);
    const long long tbase = (long long)C.t * P.nsrc * P.na + ant;
    const float2 *scale = reinterpret_cast<const float2 *>(P.scale) +
                          2 * ((long long)(P.scale_trows > 1 ? C.t : 0) * P.nchan * P.nsrc_pad + (long long)C.k * P.nsrc_pad);
    const uint32_t o_re = tc::operand_offset(4 * row + 2 * xp, 16 * chunk);
    const uint32_t o_im = tc::operand_offset(4 * QT + 4 * row + 2 * xp, 16 * chunk);
    const bool pointing = P.has_pointing != 0;
    const ChanF ch = C.ch;

    const float2 *tau0 = P.tau + tbase;
    const int na = P.na, last = P.nsrc - 1;
    auto load = [&](int it, Pre<SPC> &L) {
        const int sb = it * SPS + chunk * SPC;
        const float2 *xs = scale + 2 * sb + xp;   // zero past the last source
        if (sb + SPC - 1 <= last) {
            const float2 *p = tau0 + (size_t)sb * na;
#pragma unroll
            for (int j = 0; j < SPC; j++) L.tau[j] = p[j * na];
        } else {
#pragma unroll
            for (int j = 0; j < SPC; j++) L.tau[j] = tau0[(size_t)min(sb + j, last) * na];
        }
#pragma unroll
        for (int j = 0; j < SPC; j++) L.x[j] = xs[2 * j];
    };
    auto produce = [&](int it, const Pre<SPC> &L) {
        unsigned char *bh = C.smem + (it % NST) * STAGE_BYTES + 2 * A_BYTES, *blo = bh + B_BYTES;
        float2 a[SPC];
#pragma unroll
        for (int j = 0; j < SPC; j++) {
            a[j] = phase_sfu(L.tau[j], ch);
            if (pointing) {
                const int s = min(it * SPS + chunk * SPC + j, P.nsrc - 1);
                const float E = beam_f(P.rho[tbase + (long long)s * P.na], ch);
                a[j].x *= E;
                a[j].y *= E;
            }
        }
#pragma unroll
        for (int x = 0; x < 2; x++) {
            uint32_t h[4], l[4], hr[4], lr[4];
#pragma unroll
            for (int j = 0; j < SPC; j++) {
                const float X = x == 0 ? L.x[j].x : L.x[j].y;
                if (TF32) {
                    split_tf32(X * a[j].x, h[2 * j], l[2 * j]);
                    split_tf32(X * a[j].y, h[2 * j + 1], l[2 * j + 1]);
                } else if (FMT == FMT_F16) {
                    split_f16_rot(X * a[j].x, X * a[j].y, h[j], l[j], hr[j], lr[j]);
                } else {
                    split_bf16_rot(X * a[j].x, X * a[j].y, h[j], l[j], hr[j], lr[j]);
                }
            }
            st16(bh + o_re + 16 * x, h[0], h[1], h[2], h[3]);
            st16(blo + o_re + 16 * x, l[0], l[1], l[2], l[3]);
            if (TF32) {   // (re, im) -> (-im, re)
                st16(bh + o_im + 16 * x, h[1] ^ 0x80000000u, h[0], h[3] ^ 0x80000000u, h[2]);
                st16(blo + o_im + 16 * x, l[1] ^ 0x80000000u, l[0], l[3] ^ 0x80000000u, l[2]);
            } else {
                st16(bh + o_im + 16 * x, hr[0], hr[1], hr[2], hr[3]);
                st16(blo + o_im + 16 * x, lr[0], lr[1], lr[2], lr[3]);
            }
        }
    };
    auto no_drain = [] {};
    Pre<SPC> b0, b1;
    if (C.nstg > 0) load(0, b0);
    bool ok = true;
    if constexpr (TF32) {   // two stages per proxy fence, as the A warps (BF16 and FP16: slower)
        if (C.nstg > 1) load(1, b1);
        for (int it = 0; it < C.nstg && ok; it += 2) {
            const bool two = it + 1 < C.nstg;
            ok = wait_slot(C, it, lane, no_drain);
            if (!ok) break;
            produce(it, b0);
            if (it + 2 < C.nstg) load(it + 2, b0);
            if (two) {
                ok = wait_slot(C, it + 1, lane, no_drain);
                if (!ok) break;
                produce(it + 1, b1);
                if (it + 3 < C.nstg) load(it + 3, b1);
            }
            tc::fence_async_smem();
            tc::mbar_arrive(&C.full[it % NST]);
            if (two) tc::mbar_arrive(&C.full[(it + 1) % NST]);
        }
    } else {
        for (int it = 0; it < C.nstg && ok; it += 2) {
            for (int u = 0; u < 2 && ok && it + u < C.nstg; u++) {
                Pre<SPC> &use = u ? b1 : b0, &next = u ? b0 : b1;
                if (it + u + 1 < C.nstg) load(it + u + 1, next);
                ok = wait_slot(C, it + u, lane, no_drain);
                if (ok) {
                    produce(it + u, use);
                    tc::fence_async_smem();
                    tc::mbar_arrive(&C.full[(it + u) % NST]);
                }
            }
        }
    }
    if (!ok) *(volatile int *)C.abort_flag = 1;
}

// Warp 12, one thread: the MMAs of each stage into the current segment's
// TMEM buffer; commits free the stage and, at a segment's end, the buffer.
template <int FMT>
__device__ __forceinline__ void role_mma(const Cta &C) {
    constexpr bool TF32 = FMT == FMT_TF32;
    const uint32_t idesc =
        tc::instr_desc(TF32 ? tc::kFmtTF32 : FMT == FMT_F16 ? tc::kFmtF16 : tc::kFmtBF16, PT, NB);
    const uint32_t sbase = tc::smem_u32(C.smem);
    for (int it = 0; it < C.nstg; it++) {
        const int g = it / SEG, b = g & 1, first = it % SEG == 0;
        if (first && g >= 2 && !tc::mbar_wait(&C.seg_empty[b], ((g >> 1) - 1) & 1, C.abort_flag, C.P.wait_ns)) {
            *(volatile int *)C.abort_flag = 1;
            break;
        }
        const int slot = it % NST;
        if (!tc::mbar_wait(&C.full[slot], (it / NST) & 1, C.abort_flag, C.P.wait_ns)) {
            *(volatile int *)C.abort_flag = 1;
            break;
        }
        tc::tc_fence_after();
        const uint32_t sb = sbase + slot * STAGE_BYTES;
        const uint64_t ah = tc::smem_desc(sb), alo = tc::smem_desc(sb + A_BYTES);
        const uint64_t bh = tc::smem_desc(sb + 2 * A_BYTES), bl = tc::smem_desc(sb + 2 * A_BYTES + B_BYTES);
        const uint32_t d = C.tmem + 256 * b;   // columns: Re S (B rows 0-127), Im S (rows 128-255)
        if (TF32) {
            tc::mma_tf32(d, alo, bh, idesc, !first);
            tc::mma_tf32(d, ah, bl, idesc, 1);
            tc::mma_tf32(d, ah, bh, idesc, 1);
        } else {
            tc::mma_bf16(d, alo, bh, idesc, !first);
            tc::mma_bf16(d, ah, bl, idesc, 1);
            tc::mma_bf16(d, ah, bh, idesc, 1);
        }
        tc::mma_commit(&C.empty[slot]);
        if (it % SEG == SEG - 1 || it == C.nstg - 1) tc::mma_commit(&C.seg_full[b]);
    }
    // every MMA this thread issued must have completed before the block frees
    // the TMEM they write and the shared memory they read, also when the
    // block gave up early (the drain's own limit, not the wait limit)
    tc::mma_commit(C.drained);
    tc::mbar_wait_plain(C.drained, 0, tc::kWaitLimitNs);
}

template <int FMT, bool WRITE>
__global__ void __launch_bounds__(THREADS, 1) k_split(const SplitParams P) {
    constexpr bool TF32 = FMT == FMT_TF32;
    constexpr int SPS = Item<TF32>::SPS;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t full[NST], empty[NST], seg_full[2], seg_empty[2], drained;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag, sLast;
    __shared__ double red[THREADS / 32];

    if (inputs_bad(P.status)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x % P.ntiles;
    const int rest = blockIdx.x / P.ntiles;
    const int k = rest % P.nchan;
    const int t = rest / P.nchan;
    const int2 tl = P.tiles[tile];
    const int nstg = (P.nsrc + SPS - 1) / SPS;

    if (tid == 0) {
        for (int i = 0; i < NST; i++) {
            tc::mbar_init(&full[i], NPROD);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; i++) {
            tc::mbar_init(&seg_full[i], 1);
            tc::mbar_init(&seg_empty[i], NDRAIN);
        }
        tc::mbar_init(&drained, 1);
        abort_flag = 0;
        tc::fence_async_smem();
    }
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const Cta C{P, smem, full, empty, seg_full, seg_empty, &drained, &abort_flag, tmem_base, t, k, tl.x, nstg,
                (nstg + SEG - 1) / SEG, (uint32_t)tl.y, P.chan[k]};
    double chi = 0.0;
    if (warp < NDRAIN / 32) {
        tc::regs_inc<Regs<TF32>::A>();
        chi = role_a<FMT, WRITE>(C, tid, warp, lane);
    } else if (warp < NPROD / 32) {
        tc::regs_dec<Regs<TF32>::B>();
        role_b<FMT>(C, warp, lane);
    } else {
        tc::regs_dec<REGS_MMA>();
        if (warp == NPROD / 32 && lane == 0) role_mma<FMT>(C);
    }
    const uint32_t tmem = tmem_base;

    // ---------------------------------------------------------------- teardown
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
    if (WRITE) return;
    // chi^2: block sum, one partial per block, the last block sums them in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) chi += __shfl_down_sync(0xffffffffu, chi, o);
    if (lane == 0) red[warp] = chi;
    __syncthreads();
    if (tid == 0) {
        double b = 0.0;
        for (int i = 0; i < THREADS / 32; i++) b += red[i];
        P.partials[blockIdx.x] = b;
        __threadfence();
        const unsigned ticket = atomicAdd(P.counter, 1u);
        sLast = ticket == gridDim.x - 1;
    }
    __syncthreads();
    if (!sLast) return;
    __threadfence();
    double s = 0.0;
    for (int i = tid; i < (int)gridDim.x; i += THREADS) s += __ldcg(&P.partials[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __syncthreads();
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (tid == 0) {
        double tot = 0.0;
        for (int i = 0; i < THREADS / 32; i++) tot += red[i];
        if (P.status->err[EC_RUN] == 0) *P.result = tot;
        *P.counter = 0u;
    }
}

// Per-source factors of the B operand for each (t, k): the Stokes vector
// times the spectral factor (nu/nu_ref)^alpha (eq. 2) and, without pointing
// errors, times the beam of both antennas E_s^2 (eq. 4; the same for every
// antenna). out [trows][nchan][nsrc_pad][4], zero for s >= nsrc.
// FP16 split: B = X A with |A| <= 1 must stay below the FP16 maximum (65504)
// with room for the rounding of its high part.
constexpr float kF16Limit = 6.0e4f;
__global__ void k_split_scales(int nsrc, int nsrc_pad, int nchan, int trows, int na, const ChanF *chan,
                               const float *stokes, const float *alpha, const float *rho, int pointing, float4 *out,
                               int f16, DevStatus *st) {
    const long long n = (long long)trows * nchan * nsrc_pad;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(i % nsrc_pad);
        const long long r = i / nsrc_pad;
        const int k = (int)(r % nchan);
        const int t = (int)(r / nchan);
        if (s >= nsrc) {
            out[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const ChanF ch = chan[k];
        float f = exp2f(2.0f * alpha[s] * ch.hlr);
        if (!pointing) {
            const float E = beam_f(rho[(long long)s * na], ch);   // timestep 0, any antenna
            f *= E * E;
        }
        const float4 sv = reinterpret_cast<const float4 *>(stokes)[(long long)t * nsrc + s];
        const float4 o = make_float4(sv.x * f, sv.y * f, sv.z * f, sv.w * f);
        out[i] = o;
        if (f16 && !(fmaxf(fmaxf(fabsf(o.x), fabsf(o.y)), fmaxf(fabsf(o.z), fabsf(o.w))) <= kF16Limit)) {
            atomicOr(&st->err[EC_MODE], EB_F16);
            atomicMin(&st->first_bad[EC_MODE], (long long)s);
        }
    }
}

// Split mode takes point sources only: flags any Gaussian source.
__global__ void k_check_points(int nsrc, const float *gauss, DevStatus *st) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsrc && gauss[4 * s + 3] != 0.f) {
        atomicOr(&st->err[EC_MODE], EB_RANGE);
        atomicMin(&st->first_bad[EC_MODE], (long long)s);
    }
}

}  // namespace split

// Tile plan. Antennas fall into groups of QT = 32 (the last one ragged); a
// tile pairs one column group c (the MMA's N side) with up to four row groups
// (its M = 128 rows). S_X is Hermitian for real X (S_X[q, p] = conj S_X[p, q]),
// so each unordered pair of distinct groups {a, b} is computed once, as rows
// of a against column group b or the reverse, in the tiles of the group that
// owns the pair, and each group's own pairs p < q in one tile whose rows
// include the column group itself. Group c with o_c owned pairs needs
// ceil((o_c + 1) / 4) tiles. Each group is given a budget of t_c tiles, so at
// most 4 t_c - 1 owned pairs: the pairs can be shared out within the budgets
// iff every set of k groups can hold the k (k - 1) / 2 pairs among them, and
// the k groups of smallest budget are the tightest set; the budgets start at
// one tile and the smallest is raised until that holds. The pairs are then
// shared out along augmenting paths (a full group passes one of its pairs
// on to the pair's other group). 256 antennas (8 groups): 9 tiles, against
// the 12 of a plan of 128-antenna row blocks against 32-antenna column blocks,
// whose tiles on the diagonal hold half as many baselines.
// Tile encoding: x = c, y = row groups (8 bits each, slot 0 lowest, 0xff empty).
std::vector<int2> split_tiles(int na) {
    using split::QT;
    std::vector<int2> out;
    if (na < 2) return out;
    const int G = (na + QT - 1) / QT;
    std::vector<int> budget(G, 1), idx(G);
    for (;;) {
        for (int c = 0; c < G; c++) idx[c] = c;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return budget[a] < budget[b]; });
        long long held = 0;
        bool ok = true;
        for (int k = 1; k <= G && ok; k++) {
            held += 4 * budget[idx[k - 1]] - 1;
            ok = held >= (long long)k * (k - 1) / 2;
        }
        if (ok) break;
        budget[idx[0]]++;
    }
    // own[a * G + b]: group a owns the pair {a, b}
    std::vector<char> own((size_t)G * G, 0);
    std::vector<int> nown(G, 0), from(G);
    auto spare = [&](int v) { return nown[v] < 4 * budget[v] - 1; };
    for (int a = 0; a < G; a++)
        for (int b = a + 1; b < G; b++) {
            const int first = nown[a] - 4 * budget[a] <= nown[b] - 4 * budget[b] ? a : b, second = a + b - first;
            if (spare(first) || spare(second)) {
                const int v = spare(first) ? first : second;
                own[(size_t)v * G + (a + b - v)] = 1;
                nown[v]++;
                continue;
            }
            // breadth-first search from a and b over "v passes a pair {v, w} to w"
            std::fill(from.begin(), from.end(), -2);
            std::vector<int> queue{a, b};
            from[a] = from[b] = -1;
            int end = -1;
            for (size_t h = 0; h < queue.size() && end < 0; h++) {
                const int v = queue[h];
                for (int w = 0; w < G && end < 0; w++)
                    if (own[(size_t)v * G + w] && from[w] == -2) {
                        from[w] = v;
                        if (spare(w)) end = w;
                        else queue.push_back(w);
                    }
            }
            if (end < 0) return {};   // cannot happen once the budgets pass the test above
            nown[end]++;
            int w = end;
            for (; from[w] >= 0; w = from[w]) {   // move {from[w], w} to w along the path
                own[(size_t)from[w] * G + w] = 0;
                own[(size_t)w * G + from[w]] = 1;
            }
            own[(size_t)w * G + (a + b - w)] = 1;   // the path's start takes the new pair
        }
    for (int c = 0; c < G; c++) {
        std::vector<int> rows{c};
        for (int w = 0; w < G; w++)
            if (own[(size_t)c * G + w]) rows.push_back(w);
        for (size_t i = 0; i < rows.size(); i += 4) {
            uint32_t packed = 0xffffffffu;
            for (size_t j = 0; j < 4 && i + j < rows.size(); j++)
                packed = (packed & ~(0xffu << (8 * j))) | ((uint32_t)rows[i + j] << (8 * j));
            out.push_back(make_int2(c, (int)packed));
        }
    }
    return out;
}

extern "C" int32_t rime_split_tiles(int32_t na, int32_t *out, int32_t cap) {
    if (na < 2 || na > 4096 || cap < 0 || (cap > 0 && !out)) return -1;
    const std::vector<int2> tl = split_tiles(na);
    for (int i = 0; i < (int)tl.size() && i < cap; i++) {
        out[5 * i] = tl[i].x;
        for (int j = 0; j < 4; j++) {
            const int g = ((uint32_t)tl[i].y >> (8 * j)) & 0xff;
            out[5 * i + 1 + j] = g == 0xff ? -1 : g;
        }
    }
    return (int32_t)tl.size();
}

cudaError_t launch_split(rime_ctx *c, bool write, void *vis_out, double *result) {
    using namespace split;
    cudaError_t e;
    if (!c->d_stiles) {
        std::vector<int2> tl = split_tiles(c->dims.na);
        Alloc alloc{c};
        e = alloc((void **)&c->d_stiles, tl.size() * sizeof(int2));
        if (e != cudaSuccess) return e;
        e = cudaMemcpy(c->d_stiles, tl.data(), tl.size() * sizeof(int2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
        c->nstiles = (int)tl.size();
    }
    const long long blocks = (long long)c->dims.ntime * c->dims.nchan * c->nstiles;
    if (blocks == 0) return cudaSuccess;
    if (!write && (size_t)blocks > c->spart_cap) {
        if (c->d_spart) cudaFree(c->d_spart);
        c->d_spart = nullptr;
        c->spart_cap = 0;
        Alloc alloc{c};
        e = alloc((void **)&c->d_spart, (size_t)blocks * sizeof(double));
        if (e != cudaSuccess) return e;
        c->spart_cap = (size_t)blocks;
    }
    if (!c->d_scounter) {
        Alloc alloc{c};
        e = alloc((void **)&c->d_scounter, sizeof(unsigned));
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(c->d_scounter, 0, sizeof(unsigned), c->stream);
        if (e != cudaSuccess) return e;
    }
    e = reset_status_class(c, EC_MODE);
    if (e != cudaSuccess) return e;
    const int trows = c->time_varying ? c->dims.ntime : 1;
    const int nsrc_pad = (c->nsrc + 7) / 8 * 8;
    const size_t nscale = (size_t)trows * c->dims.nchan * nsrc_pad;
    if (nscale > c->sscale_cap) {
        if (c->d_sscale) cudaFree(c->d_sscale);
        c->d_sscale = nullptr;
        c->sscale_cap = 0;
        Alloc alloc{c};
        e = alloc((void **)&c->d_sscale, nscale * sizeof(float4));
        if (e != cudaSuccess) return e;
        c->sscale_cap = nscale;
    }
    if (c->nsrc > 0) {
        k_check_points<<<(c->nsrc + 255) / 256, 256, 0, c->stream>>>(c->nsrc, (const float *)c->d_gauss, c->d_status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int nb = (int)std::min<size_t>((nscale + 255) / 256, 4096);
        k_split_scales<<<nb, 256, 0, c->stream>>>(c->nsrc, nsrc_pad, c->dims.nchan, trows, c->dims.na,
                                                  reinterpret_cast<const ChanF *>(c->d_chan),
                                                  reinterpret_cast<const float *>(c->d_stokes),
                                                  reinterpret_cast<const float *>(c->d_alpha),
                                                  reinterpret_cast<const float *>(c->d_rho), c->has_pointing,
                                                  reinterpret_cast<float4 *>(c->d_sscale),
                                                  c->tc_mode == RIME_TC_SPLIT_F16, c->d_status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    SplitParams P{};
    P.na = c->dims.na;
    P.ntime = c->dims.ntime;
    P.nchan = c->dims.nchan;
    P.nsrc = c->nsrc;
    P.ntiles = c->nstiles;
    P.nbl = c->nbl;
    P.has_gains = c->has_gains;
    P.has_weight = c->has_weight;
    P.has_pointing = c->has_pointing;
    P.tiles = c->d_stiles;
    P.chan = reinterpret_cast<const ChanF *>(c->d_chan);
    P.tau = reinterpret_cast<const float2 *>(c->d_tau);
    P.rho = reinterpret_cast<const float *>(c->d_rho);
    P.scale = reinterpret_cast<const float *>(c->d_sscale);
    P.scale_trows = trows;
    P.nsrc_pad = nsrc_pad;
    P.gains = reinterpret_cast<const float2 *>(c->d_gains);
    P.data = reinterpret_cast<const float2 *>(c->d_data);
    P.weight = reinterpret_cast<const float *>(c->d_weight);
    P.vis_out = reinterpret_cast<float2 *>(vis_out);
    P.partials = c->d_spart;
    P.counter = c->d_scounter;
    P.result = result;
    P.status = c->d_status;
    P.wait_ns = c->wait_ns ? c->wait_ns : tc::kWaitLimitNs;
    auto go = [&](auto kernel) -> cudaError_t {
        // the warpgroup register budgets assume the block is launched with
        // exactly REGS_LAUNCH registers per thread; never launch otherwise
        cudaFuncAttributes fa;
        cudaError_t e2 = cudaFuncGetAttributes(&fa, kernel);
        if (e2 != cudaSuccess) return e2;
        if (fa.numRegs != REGS_LAUNCH) return cudaErrorInvalidConfiguration;
        e2 = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        if (e2 != cudaSuccess) return e2;
        kernel<<<(unsigned)blocks, THREADS, SMEM_BYTES, c->stream>>>(P);
        return cudaGetLastError();
    };
    if (c->tc_mode == RIME_TC_SPLIT_TF32)
        return write ? go(k_split<FMT_TF32, true>) : go(k_split<FMT_TF32, false>);
    if (c->tc_mode == RIME_TC_SPLIT_F16)
        return write ? go(k_split<FMT_F16, true>) : go(k_split<FMT_F16, false>);
    return write ? go(k_split<FMT_BF16, true>) : go(k_split<FMT_BF16, false>);
}

}  // namespace rime
