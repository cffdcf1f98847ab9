// The tcgen05 slice product of the emulated FP64 product (the persistent
// slice_gemm kernels), shared by the host code in emulated.cu and the two
// translation units that instantiate it per slice format and slice count
// (slice_gemm_bf16.cu, slice_gemm_fp8.cu).  The slice count is a template
// parameter: the MMA issue loop then has no runtime branch between MMAs, and
// the tensor pipe stays fed.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"

namespace emu {

constexpr int BM = 128, BN = 64;  // output tile rows and (at most) columns
constexpr int KB_BYTES = 64;       // one K-block of one slice row: 32 BF16 or 64 FP8 values

// Slice formats.  BF16 holds balanced base-2^7 digits (|d| <= 64, 8-bit
// significand); FP8-E4M3 holds balanced base-2^5 digits (|d| <= 16: every
// integer up to 16 in magnitude has at most 4 significant bits).
__host__ __device__ constexpr int fmt_beta(int kind) { return kind == MM_SLICE_FP8E4M3 ? 5 : 7; }
__host__ __device__ constexpr int fmt_esize(int kind) { return kind == MM_SLICE_FP8E4M3 ? 1 : 2; }
__host__ __device__ constexpr int fmt_bke(int kind) { return KB_BYTES / fmt_esize(kind); }
// K-blocks over which one slice pair's products (each at most 2^(2 beta - 2) in
// magnitude) sum to an integer FP32 holds exactly (<= 2^24).
__host__ __device__ constexpr int fmt_pair_blocks(int kind) {
    return (1 << (26 - 2 * fmt_beta(kind))) / fmt_bke(kind);
}
// Most slices per format: TMEM holds 512 FP32 columns, one accumulator per
// diagonal; 8 diagonals of 64 columns fill it, and FP8-E4M3 goes on to 10
// diagonals of 32 columns.
__host__ __device__ constexpr int fmt_max_slices(int kind) { return kind == MM_SLICE_FP8E4M3 ? 10 : 8; }
// Output tile width for s slices: 64 columns per diagonal up to 8 slices, 32
// beyond (so s accumulators still fit TMEM's 512 columns).  Up to 8 slices a
// narrow tile of 32 columns is the other choice (half the padding on narrow
// products, at the N = 64 MMA rate); the autotuner picks between the two.
__host__ __device__ constexpr int slice_bn(int s) { return s > 8 ? 32 : BN; }
__host__ __device__ constexpr bool slice_bn_ok(int s, int bn) { return bn == 32 || (bn == BN && s <= 8); }
// Launch-wide constants of the slice product, functions of the slice format
// and count only (so the kernel, templated on both, has them at compile time):
// a stage holds one K-block (64 bytes per slice row) of all s slices of A and
// B; up to 4 stages fit the shared memory; an exact chunk is the exact length
// of diagonal s - 1; TMEM is allocated in powers of two >= 32 columns.
constexpr int kSmemLimit = 232448;  // opt-in dynamic shared memory per block on sm_103
__host__ __device__ constexpr uint32_t slice_stage_bytes(int s, int bn) { return (uint32_t)s * (BM + bn) * KB_BYTES; }
__host__ __device__ constexpr int slice_stages(int s, int bn) {
    return (int)((kSmemLimit - 2048) / slice_stage_bytes(s, bn)) < 4 ? (int)((kSmemLimit - 2048) / slice_stage_bytes(s, bn))
                                                                      : 4;
}
__host__ __device__ constexpr int slice_chunk_blocks(int kind, int s) {
    return fmt_pair_blocks(kind) / s > 1 ? fmt_pair_blocks(kind) / s : 1;
}
__host__ __device__ constexpr uint32_t slice_tmem_cols(int s, int bn) {
    return (uint32_t)(s * bn <= 32    ? 32
                      : s * bn <= 64  ? 64
                      : s * bn <= 128 ? 128
                      : s * bn <= 256 ? 256
                                      : 512);
}
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;

// Everything one split of A needs (one problem).
struct SplitA {
    int64_t N, P, lda, Nr, Pp;
    const double *A;
    int s;
    int32_t *ea;
    unsigned char *slices;  // [s][Nr][Pp] elements of the slice format (the kernels' template parameter)
};

// Everything the column split of B needs (one problem).
struct SplitB {
    int64_t P, M, ldb, Mr, Pp;
    const double *B;
    int s;
    unsigned long long *colmax;  // zeroed before col_max runs
    int32_t *fb;
    unsigned char *slices;  // [s][Mr][Pp] elements of the slice format
};

struct EmuParams {
    int64_t N, P, M;
    int s;
    int tiles_m, tiles_n;
    const int32_t *ea, *fb;
    double *C;
    int64_t ldc;
    int *status;
};

__device__ __forceinline__ void raise_status(int *status, int code) {
    if (status) atomicOr(status, code);
}

// RN(W) * 2^E for the exact signed 128-bit integer W = (hi, lo), built from
// integer operations only (the FP64 pipe of this part is too slow to spend per
// output): W is rounded to a 53-bit significand, ties to even, with a sticky
// bit for everything below; the scaling by 2^E is exact unless the result
// leaves the normal range -- past the largest double it is +-inf, below the
// smallest normal it is rounded once more to the subnormal grid (ties to
// even), exactly as rounding to double and then scaling by 2^E does.
__device__ __forceinline__ double int128_scaled_to_double(int64_t hi, uint64_t lo, int E) {
    const bool neg = hi < 0;
    uint64_t uh = (uint64_t)hi, ul = lo;
    if (neg) {
        ul = ~ul + 1;
        uh = ~uh + (ul == 0 ? 1 : 0);
    }
    if ((uh | ul) == 0) return 0.0;
    const uint64_t sign = neg ? (1ull << 63) : 0ull;
    // Normalise so the leading one sits at bit 127 of (h, l).
    const int lz = uh ? __clzll((long long)uh) : 64 + __clzll((long long)ul);
    uint64_t h, l;
    if (lz >= 64) {
        h = ul << (lz - 64);
        l = 0;
    } else if (lz > 0) {
        h = (uh << lz) | (ul >> (64 - lz));
        l = ul << lz;
    } else {
        h = uh;
        l = ul;
    }
    // 53-bit significand, guard bit, sticky bit.
    uint64_t m = h >> 11;
    const bool guard = (h >> 10) & 1ull, sticky = (h & 0x3FFull) != 0 || l != 0;
    int msb = 127 - lz;  // W's leading bit has weight 2^msb
    if (guard && (sticky || (m & 1ull))) {
        if (++m == (1ull << 53)) {
            m >>= 1;
            ++msb;
        }
    }
    const int biased = msb + E + 1023;  // exponent field of RN(W) 2^E
    if (biased >= 2047) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
    if (biased >= 1)
        return __longlong_as_double((long long)(sign | ((uint64_t)biased << 52) | (m & ((1ull << 52) - 1))));
    // Subnormal: m 2^(msb - 52 + E) on the grid of 2^-1074, `shift` low bits dropped.
    const int shift = 1 - biased;
    if (shift > 53) return __longlong_as_double((long long)sign);
    uint64_t q = m >> shift;
    const uint64_t rem = m & ((1ull << shift) - 1), half = 1ull << (shift - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
    return __longlong_as_double((long long)(sign | q));  // q = 2^52 carries into the exponent field
}

// Tile of CTA `id` in a tiles_m x tiles_n grid, in runs of 8 tile-rows so that
// consecutive CTAs share B slices in L2.
__device__ __forceinline__ void tile_of(int64_t id, int tiles_m, int tiles_n, int &tm, int &tn) {
    const int64_t per_group = 8 * (int64_t)tiles_n;
    const int64_t group = id / per_group, first_m = group * 8;
    const int gsize = (int)min((int64_t)tiles_m - first_m, (int64_t)8);
    tm = (int)(first_m + (id % per_group) % gsize);
    tn = (int)((id % per_group) / gsize);
}

// Accumulator d holds d + 1 slice pairs, so its exact length is
// L_d = pair_blocks / (d + 1) K-blocks, a whole number r_d = floor(L_d / CB) of
// chunks of CB = L_(s-1) K-blocks: at each chunk end only the accumulators
// whose periods are complete are read out (plus all of them at the tile's last
// chunk), which cuts the TMEM traffic of the drains by about a third for 8
// slices.  Diagonals 2j and 2j + 1 share one period, that of 2j + 1 (the
// shorter, so both stay exact): they are written by the same N = 128 MMAs
// (see slice_tiles) and must start over together.  The countdowns live in one
// register (64 bits: 4 bits per diagonal, up to 10).
constexpr int kMaxDiag = 10;
__device__ __forceinline__ uint64_t drain_periods(int CB, int pair_blocks) {
    uint64_t R = 0;
#pragma unroll
    for (int d = 0; d < kMaxDiag; ++d) {
        const int dd = d | 1;
        R |= (uint64_t)(min(16, max(1, (pair_blocks / (dd + 1)) / CB)) - 1) << (4 * d);
    }
    return R;
}
// Diagonals due at this chunk end; advances the countdowns.
__device__ __forceinline__ uint32_t drain_due(uint64_t &cnt, uint64_t R, bool last) {
    uint32_t due = 0;
    uint64_t nc = 0;
#pragma unroll
    for (int d = 0; d < kMaxDiag; ++d) {
        const uint32_t v = (uint32_t)(cnt >> (4 * d)) & 15u;
        const bool z = last || v == 0;
        due |= (uint32_t)z << d;
        nc |= (uint64_t)(z ? (uint32_t)(R >> (4 * d)) & 15u : v - 1) << (4 * d);
    }
    cnt = nc;
    return due;
}

// d = a * b + c with a 64-bit c (one multiply-add of the integer pipe).
__device__ __forceinline__ int64_t mad_wide(int32_t a, int32_t b, int64_t c) {
    int64_t d;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// One output tile of one problem: its slice tensor maps (kernel parameters or
// entries of a grouped launch's table in global memory), parameters and place.
struct TileJob {
    const CUtensorMap *tmA, *tmB;
    EmuParams p;
    int tm, tn;
};

// Persistent slice product: CTA b takes tiles b, b + gridDim.x, ... of the
// launch (Tiles::get resolves one).  The TMA warp, the MMA warp and the
// epilogue warps walk the same tile sequence; stage and accumulator barrier
// phases run on across tiles, so the loads of the next tile start while the
// last chunk of the current one is in the tensor pipe, and its MMAs start as
// soon as the epilogue has read the accumulators out -- the final rounding and
// the stores of C overlap them.  The slice count kS is a template parameter,
// and with it the stage count, the exact chunk and the TMEM columns; so is
// the tile width kBN (64, or 32).
template <bool kFP8, int kS, int kBN, class Tiles>
__device__ __forceinline__ void slice_tiles(const Tiles &tiles, int64_t total, const EmuParams &c,
                                            bool maps_in_global) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bars[2 * 8 + 3];
    __shared__ uint32_t tmem_slot;
    if ((int64_t)blockIdx.x >= total) return;  // whole CTA, before any barrier
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int KIND = kFP8 ? MM_SLICE_FP8E4M3 : MM_SLICE_BF16;
    constexpr int bke = fmt_bke(KIND), pair_blocks = fmt_pair_blocks(KIND);
    static_assert(kS >= 1 && kS <= fmt_max_slices(KIND), "1 to 8 BF16 or 1 to 10 FP8-E4M3 slices");
    constexpr int s = kS;
    static_assert(slice_bn_ok(kS, kBN), "64-column tiles up to 8 slices, 32-column tiles for any count");
    constexpr int TBN = kBN;      // tile width
    constexpr int CPT = TBN / 2;  // columns each epilogue thread drains and rounds
    constexpr int S = slice_stages(s, TBN), CB = slice_chunk_blocks(KIND, s);
    constexpr uint32_t a_bytes = (uint32_t)s * BM * KB_BYTES, b_bytes = (uint32_t)s * TBN * KB_BYTES;
    constexpr uint32_t stage_bytes = slice_stage_bytes(s, TBN), tmem_cols = slice_tmem_cols(s, TBN);
    static_assert(a_bytes + b_bytes == stage_bytes, "stage layout");
    uint64_t *full = bars, *empty = bars + 8, *acc_full = bars + 16, *acc_empty = bars + 17, *mma_done = bars + 18;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mmdev::mbar_init(&full[i], 1);
            mmdev::mbar_init(&empty[i], 1);
        }
        mmdev::mbar_init(acc_full, 1);
        mmdev::mbar_init(acc_empty, kEpiWarps);
        mmdev::mbar_init(mma_done, 1);
        mmdev::fence_mbar_init();
    }
    if (warp == 1) {
        mmdev::tmem_alloc(&tmem_slot, tmem_cols);
        mmdev::tmem_relinquish();
    }
    mmdev::tc_fence_before();
    __syncthreads();
    mmdev::tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;  // K-blocks loaded so far, over all tiles of this CTA
            bool ok = true;
            for (int64_t id = blockIdx.x; id < total && ok; id += gridDim.x) {
                TileJob j;
                tiles.get(id, j);
                if (maps_in_global) {  // the grouped table is rewritten in place between launches
                    mmdev::tmap_acquire(j.tmA);
                    mmdev::tmap_acquire(j.tmB);
                }
                mmdev::prefetch_tmap(j.tmA);
                mmdev::prefetch_tmap(j.tmB);
                const int nkb = (int)((j.p.P + bke - 1) / bke);
                const int32_t m0 = j.tm * BM, n0 = j.tn * TBN;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const uint32_t st = it % S, use = it / S;
                    if (use > 0 && !mmdev::mbar_wait(&empty[st], (use - 1) & 1u)) {
                        raise_status(c.status, mm::kStatusTimeoutTma);
                        ok = false;
                        break;
                    }
                    uint8_t *sa = smem + (size_t)st * stage_bytes;
                    mmdev::mbar_arrive_expect_tx(&full[st], stage_bytes);
                    mmdev::tma_load_3d(sa, j.tmA, &full[st], kb * bke, m0, 0);
                    mmdev::tma_load_3d(sa + a_bytes, j.tmB, &full[st], kb * bke, n0, 0);
                }
            }
            // Wait (bounded) for the last load into each stage, so no copy is in flight at exit.
            for (uint32_t k = it > (uint32_t)S ? it - S : 0u; k < it; ++k)
                (void)mmdev::mbar_wait(&full[k % S], (k / S) & 1u);
        }
    } else if (warp == 1) {
        // The whole warp runs the issue loop; each MMA and commit is issued by one
        // elected lane.  Descriptors are the stage's base descriptors plus
        // compile-time offsets (the start-address field cannot carry: shared
        // addresses stay below 2^18).  B's slices sit one after another in the
        // stage, so one M = 128, N = 128 MMA of A slice sigma against B slices
        // tau and tau + 1 adds into accumulators d = sigma + tau and d + 1,
        // which are adjacent in TMEM: the 36 pair products of 8 slices go out
        // as 20 MMAs per K-step, and the loop is fully unrolled with no branch
        // between them.  sigma = 0 writes every accumulator first, so it alone
        // carries the start-over flag.
        const uint32_t idesc = kFP8 ? mmdev::idesc_e4m3_f32(BM, TBN) : mmdev::idesc_bf16_f32(BM, TBN);
        const uint32_t idesc2 = kFP8 ? mmdev::idesc_e4m3_f32(BM, 2 * TBN) : mmdev::idesc_bf16_f32(BM, 2 * TBN);
        const uint64_t R = drain_periods(CB, pair_blocks);
        uint32_t it = 0, ev = 0;  // K-blocks consumed and chunks handed to the epilogue, over all tiles
        bool ok = true;
        for (int64_t id = blockIdx.x; id < total && ok; id += gridDim.x) {
            TileJob j;
            tiles.get(id, j);
            const int nkb = (int)((j.p.P + bke - 1) / bke);
            int kin = 0;                // K-block within the current exact chunk
            uint64_t cnt = R;
            uint32_t fresh = ~0u;  // accumulators that start over at the next chunk
            for (int kb = 0; kb < nkb; ++kb, ++it) {
                const uint32_t st = it % S, use = it / S;
                if (kin == 0 && ev > 0) {  // the accumulators must have been read out
                    ok = __all_sync(0xffffffffu, mmdev::mbar_wait(acc_empty, (ev - 1) & 1u));
                    if (!ok) break;
                    mmdev::tc_fence_after();
                }
                ok = __all_sync(0xffffffffu, mmdev::mbar_wait(&full[st], use & 1u));
                if (!ok) break;
                mmdev::tc_fence_after();
                const uint32_t a_base = mmdev::smem_u32(smem + (size_t)st * stage_bytes);
                const uint64_t da = mmdev::smem_desc_sw64(a_base), db = mmdev::smem_desc_sw64(a_base + a_bytes);
                const uint32_t fresh_now = kin == 0 ? fresh : 0u;
#pragma unroll
                for (int sg = 0; sg < s; ++sg) {
#pragma unroll
                    for (int tu = 0; tu < s - sg; tu += 2) {
                        const int d = sg + tu;
                        const uint32_t id2 = tu + 1 < s - sg ? idesc2 : idesc;  // a pair, or the last one alone
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint64_t ad = da + (uint64_t)((sg * (BM * KB_BYTES) + kk * 32) >> 4);
                            const uint64_t bd = db + (uint64_t)((tu * (TBN * KB_BYTES) + kk * 32) >> 4);
                            const uint32_t acc = (sg == 0 && kk == 0) ? (((fresh_now >> d) & 1u) ^ 1u) : 1u;
                            if (kFP8)
                                mmdev::mma_e4m3_elect(tmem + (uint32_t)(d * TBN), ad, bd, id2, acc);
                            else
                                mmdev::mma_bf16_elect(tmem + (uint32_t)(d * TBN), ad, bd, id2, acc);
                        }
                    }
                }
                mmdev::mma_commit_elect(&empty[st]);
                if (++kin == CB || kb == nkb - 1) {
                    mmdev::mma_commit_elect(acc_full);
                    fresh = drain_due(cnt, R, kb == nkb - 1);
                    ++ev;
                    kin = 0;
                }
            }
        }
        if (!ok && lane == 0) raise_status(c.status, mm::kStatusTimeoutMma);
        // Every MMA issued above has completed once mma_done flips.
        mmdev::mma_commit_elect(mma_done);
        (void)mmdev::mbar_wait(mma_done, 0);
    } else {
        const int q = warp & 3, h = (warp - 2) >> 2;
        const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(CPT * h);
        uint32_t ev = 0;
        bool ok = true;
        constexpr int hsplit = (s + 1) / 2;  // diagonals [0, hsplit) sum into whi, the rest into wlo
        constexpr int beta = fmt_beta(KIND);
        const uint64_t R = drain_periods(CB, pair_blocks);
        for (int64_t id = blockIdx.x; id < total && ok; id += gridDim.x) {
            int nchunks;
            {
                TileJob j;
                tiles.get(id, j);
                nchunks = ((int)((j.p.P + bke - 1) / bke) + CB - 1) / CB;
            }
            int64_t whi[CPT], wlo[CPT];
#pragma unroll
            for (int k = 0; k < CPT; ++k) whi[k] = wlo[k] = 0;
            uint64_t cnt = R;
            for (int ch = 0; ch < nchunks; ++ch, ++ev) {
                if (!mmdev::mbar_wait(acc_full, ev & 1u)) {
                    raise_status(c.status, mm::kStatusTimeoutEpi);
                    ok = false;
                    break;
                }
                mmdev::tc_fence_after();
                const uint32_t due = drain_due(cnt, R, ch == nchunks - 1);
                // Unrolled over the diagonals, so each one's weight is a constant and
                // its accumulator array is known: one exact conversion and one
                // 32 x 32 -> 64-bit multiply-add per value.
#pragma unroll
                for (int d = 0; d < s; ++d) {
                    if (!((due >> d) & 1u)) continue;
                    uint32_t v[CPT];
                    if constexpr (CPT == 32)
                        mmdev::tmem_ld_32x32b_x32(tbase + (uint32_t)(d * TBN), v);
                    else
                        mmdev::tmem_ld_32x32b_x16(tbase + (uint32_t)(d * TBN), v);
                    mmdev::tmem_wait_ld();
                    const int32_t weight = 1 << (d < hsplit ? beta * (hsplit - 1 - d) : beta * (s - 1 - d));
                    int64_t *acc = d < hsplit ? whi : wlo;
#pragma unroll
                    for (int k = 0; k < CPT; ++k)
                        acc[k] = mad_wide(__float2int_rn(__uint_as_float(v[k])), weight, acc[k]);
                }
                mmdev::tc_fence_before();
                __syncwarp();
                if (lane == 0) mmdev::mbar_arrive(acc_empty);
            }
            // The accumulators are free again: round and store while the next tile's MMAs
            // run (the tile is resolved again so its parameters need no registers above).
            TileJob j;
            tiles.get(id, j);
            const EmuParams &p = j.p;
            const int64_t row = (int64_t)j.tm * BM + 32 * q + lane, n0 = (int64_t)j.tn * TBN;
            if (ok && row < p.N) {
                const int e = p.ea[row];
                const int sh2 = beta * (s - hsplit);
                double *crow = p.C + row * p.ldc;
#pragma unroll
                for (int k = 0; k < CPT; k += 2) {
                    double out[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int64_t col = n0 + CPT * h + k + u;
                        const int64_t wh = whi[k + u], wl = wlo[k + u];
                        // W = wh * 2^sh2 + wl as a signed 128-bit integer.
                        uint64_t lo = sh2 ? ((uint64_t)wh << sh2) : (uint64_t)wh;
                        int64_t hi = sh2 ? (wh >> (64 - sh2)) : (wh >> 63);
                        const uint64_t lo2 = lo + (uint64_t)wl;
                        hi += (wl >> 63) + (lo2 < lo ? 1 : 0);
                        lo = lo2;
                        const int f = (col < p.M) ? p.fb[col] : 0;
                        out[u] = int128_scaled_to_double(hi, lo, e + f + 2 - beta * (s + 1));
                    }
                    const int64_t col = n0 + CPT * h + k;
                    double *dst = crow + col;
                    if (col + 1 < p.M && (((uintptr_t)dst & 15) == 0)) {
                        *reinterpret_cast<double2 *>(dst) = make_double2(out[0], out[1]);
                    } else {
                        if (col < p.M) dst[0] = out[0];
                        if (col + 1 < p.M) dst[1] = out[1];
                    }
                }
            }
        }
    }

    mmdev::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        mmdev::tc_fence_after();
        mmdev::tmem_dealloc(tmem, tmem_cols);
    }
}

struct SingleTiles {
    const CUtensorMap *tmA, *tmB;
    const EmuParams *p;
    __device__ __forceinline__ void get(int64_t id, TileJob &j) const {
        j.tmA = tmA;
        j.tmB = tmB;
        j.p = *p;
        tile_of(id, p->tiles_m, p->tiles_n, j.tm, j.tn);
    }
};

template <bool kFP8, int kS, int kBN>
__global__ void __launch_bounds__(kThreads, 1)
    slice_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const EmuParams p) {
    const SingleTiles tiles{&tmA, &tmB, &p};
    slice_tiles<kFP8, kS, kBN>(tiles, (int64_t)p.tiles_m * p.tiles_n, p, false);
}

// ------------------------------------------------------------ grouped launch
//
// Many products with one slice count in one launch per kernel.  The host
// writes a table of EmuProblem entries, four prefix arrays (per kernel, the
// first CTA of each problem) and a header with the totals into the workspace;
// each CTA finds its problem by binary search over the prefix array.  Every
// kernel strides over its units, so its grid is a fixed size independent of
// the batch: the serving loop captures the five launches once per slice
// format and count in a CUDA graph and replays it for any batch.
struct EmuProblem {  // 128-byte aligned through its tensor maps
    CUtensorMap tmA, tmB;
    EmuParams prm;
    SplitA spa;
    SplitB spb;
};

struct GroupHeader {
    int64_t count;
    int64_t units[5];  // split_rows, col_max, split_cols, slice_gemm, zero_colmax CTAs
};

enum { U_ROWS = 0, U_COLMAX = 1, U_SPLITCOLS = 2, U_TILES = 3, U_ZERO = 4 };

// Largest g in [0, count) with begin[g] <= unit.
__device__ __forceinline__ int find_problem(const int64_t *begin, int64_t count, int64_t unit) {
    int64_t lo = 0, hi = count - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= unit)
            lo = mid;
        else
            hi = mid - 1;
    }
    return (int)lo;
}

struct GroupTiles {
    const EmuProblem *tab;
    const int64_t *begin;
    int64_t count;
    __device__ __forceinline__ void get(int64_t id, TileJob &j) const {
        const int g = find_problem(begin, count, id);
        const EmuProblem &e = tab[g];
        j.tmA = &e.tmA;
        j.tmB = &e.tmB;
        j.p = e.prm;
        tile_of(id - begin[g], j.p.tiles_m, j.p.tiles_n, j.tm, j.tn);
    }
};

template <bool kFP8, int kS, int kBN>
__global__ void __launch_bounds__(kThreads, 1) group_slice_gemm_kernel(const EmuProblem *tab, const int64_t *begin,
                                                                       const GroupHeader *hdr) {
    const int64_t total = hdr->units[U_TILES];
    if (total <= 0) return;
    const GroupTiles tiles{tab, begin, hdr->count};
    const EmuParams c = tab[0].prm;  // one slice format and count per launch: the constants are common
    slice_tiles<kFP8, kS, kBN>(tiles, total, c, true);
}

// Launchers, one per slice format (defined in slice_gemm_bf16.cu and
// slice_gemm_fp8.cu): launch the instantiation for slice count s (1..8 BF16,
// 1..10 FP8-E4M3) and tile width bn (64 up to 8 slices, or 32) with the given
// grid and dynamic shared memory on st.  cudaErrorInvalidValue for an (s, bn)
// outside that range (nothing is launched); otherwise cudaSuccess, launch
// errors are left for cudaGetLastError.
cudaError_t launch_slice_gemm_bf16(int s, int bn, unsigned grid, size_t smem, cudaStream_t st, const CUtensorMap &tmA,
                                   const CUtensorMap &tmB, const EmuParams &prm);
cudaError_t launch_slice_gemm_fp8(int s, int bn, unsigned grid, size_t smem, cudaStream_t st, const CUtensorMap &tmA,
                                  const CUtensorMap &tmB, const EmuParams &prm);
cudaError_t launch_group_slice_gemm_bf16(int s, int bn, unsigned grid, size_t smem, cudaStream_t st,
                                         const EmuProblem *tab, const int64_t *begin, const GroupHeader *hdr);
cudaError_t launch_group_slice_gemm_fp8(int s, int bn, unsigned grid, size_t smem, cudaStream_t st,
                                        const EmuProblem *tab, const int64_t *begin, const GroupHeader *hdr);
// Opt every instantiation of one format into `bytes` of dynamic shared memory.
cudaError_t slice_gemm_smem_attributes_bf16(int bytes);
cudaError_t slice_gemm_smem_attributes_fp8(int bytes);

// Dispatch by slice count and tile width over the instantiations (used only by
// the two instantiating translation units).
template <bool kFP8, int kS = 1>
cudaError_t dispatch_slice_gemm(int s, int bn, unsigned grid, size_t smem, cudaStream_t st, const CUtensorMap &tmA,
                                const CUtensorMap &tmB, const EmuParams &prm) {
    if (s == kS) {
        if (bn == 32) {
            slice_gemm_kernel<kFP8, kS, 32><<<grid, kThreads, smem, st>>>(tmA, tmB, prm);
            return cudaSuccess;
        }
        if constexpr (slice_bn_ok(kS, BN)) {
            if (bn == BN) {
                slice_gemm_kernel<kFP8, kS, BN><<<grid, kThreads, smem, st>>>(tmA, tmB, prm);
                return cudaSuccess;
            }
        }
        return cudaErrorInvalidValue;
    }
    if constexpr (kS < fmt_max_slices(kFP8 ? MM_SLICE_FP8E4M3 : MM_SLICE_BF16))
        return dispatch_slice_gemm<kFP8, kS + 1>(s, bn, grid, smem, st, tmA, tmB, prm);
    return cudaErrorInvalidValue;
}

template <bool kFP8, int kS = 1>
cudaError_t dispatch_group_slice_gemm(int s, int bn, unsigned grid, size_t smem, cudaStream_t st, const EmuProblem *tab,
                                      const int64_t *begin, const GroupHeader *hdr) {
    if (s == kS) {
        if (bn == 32) {
            group_slice_gemm_kernel<kFP8, kS, 32><<<grid, kThreads, smem, st>>>(tab, begin, hdr);
            return cudaSuccess;
        }
        if constexpr (slice_bn_ok(kS, BN)) {
            if (bn == BN) {
                group_slice_gemm_kernel<kFP8, kS, BN><<<grid, kThreads, smem, st>>>(tab, begin, hdr);
                return cudaSuccess;
            }
        }
        return cudaErrorInvalidValue;
    }
    if constexpr (kS < fmt_max_slices(kFP8 ? MM_SLICE_FP8E4M3 : MM_SLICE_BF16))
        return dispatch_group_slice_gemm<kFP8, kS + 1>(s, bn, grid, smem, st, tab, begin, hdr);
    return cudaErrorInvalidValue;
}

template <bool kFP8, int kS, int kBN>
cudaError_t set_one_slice_gemm_smem(int bytes) {
    cudaError_t e = cudaFuncSetAttribute((const void *)slice_gemm_kernel<kFP8, kS, kBN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)group_slice_gemm_kernel<kFP8, kS, kBN>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

template <bool kFP8, int kS = 1>
cudaError_t set_slice_gemm_smem(int bytes) {
    cudaError_t e = set_one_slice_gemm_smem<kFP8, kS, 32>(bytes);
    if constexpr (slice_bn_ok(kS, BN))
        if (e == cudaSuccess) e = set_one_slice_gemm_smem<kFP8, kS, BN>(bytes);
    if constexpr (kS < fmt_max_slices(kFP8 ? MM_SLICE_FP8E4M3 : MM_SLICE_BF16))
        if (e == cudaSuccess) return set_slice_gemm_smem<kFP8, kS + 1>(bytes);
    return e;
}

}  // namespace emu
