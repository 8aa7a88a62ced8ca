// dense.cu -- the algebraic level expansion of Section 3.1.1 on tcgen05
// tensor cores (flag BC_DENSE).
//
// ComputePathCount multiplies by the adjacency matrix A once per level. In
// frontier form (the mask read as "not reached yet" rather than the previous
// level only), for a batch of B = 128 sources:
//     C_l[s][u] = sigma_s(u) if d(s,u) = l, else 0,
//     C_{l+1} = (C_l . A) masked to the (s, v) not reached yet,
// and the non-zero entries of C_{l+1} are sigma_s(v) for d(s,v) = l+1.
// sigma is an exact uint64, so C_l is split into 8-bit limbs
//     C_l = sum_q 2^(8q) C_l^(q),   0 <= C_l^(q) <= 255,
// and each limb matrix is multiplied on the tensor cores in bf16 with FP32
// accumulation. Both are exact: bf16 holds every integer up to 256, A is 0/1,
// and every partial sum is at most 255 * n < 2^24 (n <= 65536), which FP32
// holds exactly. The epilogue converts each limb sum back to an integer and
// carry-combines sum_q 2^(8q) acc_q in 64 bits with an overflow flag.
// Only the limbs that can be non-zero are multiplied: the previous level
// reports its largest sigma, which fixes the limb count (up to 8).
//
// GEMM tile: one CTA owns N target vertices (columns of A; N = 64, 128 or
// 256) for all 128 sources and all limbs: accumulator q (128 lanes x N
// columns of FP32) sits in TMEM columns [Nq, Nq + N). Operand tiles arrive by
// TMA (128- or 64-byte swizzle, one copy per CTA) through an S-stage
// shared-memory ring guarded by mbarriers; one thread issues tcgen05.mma; four
// warps read TMEM back. The kernels are bound by the rate at which an SM takes
// in operand bytes, so the tile is as wide as TMEM allows (more products per
// byte), and the epilogue's loads that do not depend on the MMAs are issued
// ahead of their use.
// Every wait is bounded (global timer); on expiry the kernel records an error,
// drains what it issued, frees its TMEM and returns.
//
// The epilogue writes the same state the sparse level kernel writes (sigma
// [n][128], frontier and visited words, union-frontier bits), so the sparse
// backward sweep and summaries run unchanged afterwards.
#include <cuda.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>

#include "bc_internal.cuh"
#include "dense.cuh"

namespace bcgb {
namespace {

constexpr int kDB = 128;          // sources per batch (GEMM M)
constexpr int kDW = kDB / 32;     // frontier words per vertex
constexpr int kNT = 64;           // target vertices per CTA (GEMM N) of the narrow tile
constexpr int kNW = 128;          // of the wide tile
constexpr int kNX = 256;          // of the widest tile (one CTA per SM when its accumulators take all of TMEM)
// K per pipeline stage: 64 (rows of 128 bytes of bf16, 128-byte swizzle) or
// 32 (rows of 64 bytes, 64-byte swizzle: half the bytes per stage, so twice
// the stages fit the same shared memory)
// kF8: operands in e4m3 (one byte per element, 4-bit limbs) instead of bf16.
template <int kK, bool kF8 = false>
constexpr int row_bytes() { return kF8 ? kK : 2 * kK; }
template <int kK, bool kF8 = false>
constexpr int x_tile() { return kDB * row_bytes<kK, kF8>(); }  // one limb's (or part's) operand tile
// TMEM accumulators of the backward's three parts. 2 keeps the hi products
// apart from the mid and lo ones: sums of hi parts (8 significant bits each)
// stay exact, and the mid + lo sum loses nothing to hi's magnitude. 1 sums all
// three in one accumulator (half the TMEM columns, three CTAs per SM instead
// of two, about 8% faster on G(8192, 0.05)), but the tensor core's FP32
// accumulation then drops low bits of every lo and mid product against the
// hi-sized total, a bias that pulls BC down (4.4e-6 relative over all sources
// at n = 8192) and grows with n.
constexpr int kBwdAcc = 2;
template <int kN, int kK, bool kF8 = false>
constexpr int a_tile() { return kN * row_bytes<kK, kF8>(); }  // adjacency tile of an N-vertex CTA
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}
// Bounded wait on a phase; false when the time limit passed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint64_t t0 = gtimer();
    while (!mbar_try_wait(bar, parity))
        if (gtimer() - t0 > kWaitNs) return false;
    return true;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int32_t x, int32_t y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// Shared-memory matrix descriptor: K-major tile of rows of kRB bytes (128 or
// 64) with the matching swizzle (8-row atoms of 1024 or 512 bytes); start
// address, stride between atoms (the atom's bytes), descriptor version 1,
// layout SWIZZLE_128B (code 2) or SWIZZLE_64B (code 4).
template <int kRB>
__device__ __forceinline__ uint64_t sw_desc(uint32_t saddr) {
    static_assert(kRB == 128 || kRB == 64, "stage rows are 128 or 64 bytes");
    constexpr uint32_t atom = 8u * kRB;
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(atom >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)(kRB == 128 ? 2u : 4u) << 61;
    return d;
}
// Instruction descriptor: FP32 accumulator (bits 4-5 = 1), A and B both
// K-major, M = 128, N = kN; A and B bf16 (format 1 in bits 7-9 and 10-12, for
// kind::f16) or both e4m3 (format 0, for kind::f8f6f4).
template <int kN, bool kF8 = false>
constexpr uint32_t idesc() {
    return (1u << 4) | ((kF8 ? 0u : 1u) << 7) | ((kF8 ? 0u : 1u) << 10) | ((uint32_t)(kN >> 3) << 17) |
           ((uint32_t)(kDB >> 4) << 24);
}

// One MMA over 32 bytes of K (16 bf16 or 32 e4m3 elements).
template <int kN, bool kF8 = false>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    if constexpr (kF8) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc<kN, true>()), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc<kN, false>()), "r"(acc)
            : "memory");
    }
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Epilogue inputs of 16 columns v0 .. v0 + 15 that do not depend on the MMAs:
// the frontier word of each column for this thread's warp (forward: visited
// or in frontier l; backward: in frontier l) and, backward, sigma_b(v). All
// loads are issued before any is used; columns past n read nothing.
template <bool kBwd>
__device__ __forceinline__ void epi_prefetch(int n, const uint32_t *Fl, const uint32_t *Vin, const uint64_t *sigma,
                                             int v0, int warp, int b, uint32_t (&fw)[16], uint64_t (&sv)[16]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int v = v0 + i;
        const bool in = v < n;
        const size_t wi = (size_t)(in ? v : 0) * kDW + warp;
        if constexpr (kBwd) {
            fw[i] = in ? __ldg(Fl + wi) : 0u;
            sv[i] = in ? __ldg(reinterpret_cast<const unsigned long long *>(sigma) + (size_t)(in ? v : 0) * kDB + b)
                       : 0ull;
        } else {
            fw[i] = in ? (__ldg(Vin + wi) | __ldg(Fl + wi)) : 0u;
            sv[i] = 0ull;
        }
    }
}

// kBwd = false: forward level l -> l+1 (limb sums -> exact counts).
// kBwd = true:  backward level l: the three bf16 parts of the masked c rows of
//               level l+1 (rows xrow0 .. xrow0 + 383 of X) times A give
//               sum_w c_s(w) over the successors; the epilogue forms delta and
//               c for level l, adds the batch's delta to BC (FP64, fixed
//               order) and, when write_next, writes the split c rows of level l
//               at rows xout .. xout + 383.
//
// kT threads (128 or 256): warp w reads TMEM lanes 32 (w % 4) .. + 31 (the
// sources of that quarter) and, with 256 threads, warps 0-3 take the first
// half of the tile's columns in the epilogue and warps 4-7 the second half.
template <bool kBwd, int kN, int kK, int kT, bool kF8 = false>
__global__ void __launch_bounds__(kT, 1)
    k_dense_level(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmA, const DenseParams p,
                  const int l, const int nl, const int stages, const int write_next) {
    extern __shared__ unsigned char dsm_raw[];
    unsigned char *dsm = reinterpret_cast<unsigned char *>(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
    constexpr int kRB = row_bytes<kK, kF8>();
    constexpr int kXTile = x_tile<kK, kF8>();
    const int stage_bytes = nl * kXTile + a_tile<kN, kK, kF8>();
    uint64_t *bars = reinterpret_cast<uint64_t *>(dsm + (size_t)stages * stage_bytes);
    uint64_t *full = bars;
    uint64_t *empty = bars + stages;
    uint64_t *done = bars + 2 * stages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * stages + 1);
    __shared__ uint32_t s_err;

    const int tid = threadIdx.x, lane = tid & 31;
    const int warp = (tid >> 5) & 3;                  // TMEM lane quarter = source word
    constexpr int kGroups = kT / 128;                 // column groups of the epilogue
    constexpr int kCols = kN / kGroups;               // columns of each group
    const int cbeg = (tid >> 7) * kCols;              // this thread's first column
    // CTA -> (batch, 64-vertex tile): groups of p.group batches walk the
    // vertex tiles together, so each adjacency tile is read by p.group
    // batches in turn while it is in L2, and each batch's limb rows stay hot
    const int NV = p.npad / kN;
    const int per = p.group * NV;
    const int bg = blockIdx.x / per;
    const int gbase = bg * p.group;
    const int gsz = min(p.group, p.nactive - gbase);
    const int within = blockIdx.x - bg * per;
    const int vt = within / gsz;
    const int bb = p.blist[gbase + (within - vt * gsz)];
    const int v0 = vt * kN;
    uint64_t *const sigma = p.sigma + (size_t)bb * p.sig_stride;
    uint32_t *const Fb = p.F + (size_t)bb * p.f_stride;
    uint32_t *const Vb = p.V + (size_t)bb * p.v_stride;
    uint32_t *const ufb = p.ufr + (size_t)bb * p.u_stride;
    const int nbv = p.nbs[bb];
    int xin = 0, xout = 0;
    if constexpr (kBwd) {  // the two split-row blocks of this batch alternate from its deepest level down
        const int L = p.depth[bb];
        xin = ((L - 1 - l) & 1) ? 3 * kDB : 0;
        xout = 3 * kDB - xin;
    }
    const int xrow0 = bb * (kF8 ? 2 * p.xrows : p.xrows) + xin;  // e4m3 rows: npad bytes, two per bf16 row
    const int nk = p.npad / kK;
    // the backward keeps kBwdAcc accumulators for its three parts (see kBwdAcc)
    const int nacc = kBwd ? kBwdAcc : nl;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(nacc * kN)) ncols <<= 1;

    if (tid == 0) {
        s_err = 0u;
        for (int s = 0; s < stages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (tid == 0) {
        // producer: TMA the nl limb tiles and the adjacency tile of each K step
        int issued = 0;
        for (int it = 0; it < nk; ++it) {
            const int s = it % stages;
            if (it >= stages && !mbar_wait(empty + s, ((it / stages) - 1) & 1)) {
                atomicOr(&s_err, 1u);
                break;
            }
            unsigned char *st = dsm + (size_t)s * stage_bytes;
            mbar_expect_tx(full + s, (uint32_t)stage_bytes);
            for (int q = 0; q < nl; ++q)
                tma_load_2d(st + (size_t)q * kXTile, &tmX, it * kK, xrow0 + q * kDB, full + s);
            tma_load_2d(st + (size_t)nl * kXTile, &tmA, it * kK, v0, full + s);
            issued = it + 1;
        }
        // drain: every issued load must have landed before shared memory is released
        for (int it = (issued > stages ? issued - stages : 0); it < issued; ++it)
            if (!mbar_wait(full + (it % stages), (it / stages) & 1)) atomicOr(&s_err, 2u);
    } else if (tid == 32) {
        // MMA issuer: D_q += X_q . A^T over the K steps, 4 instructions (K = 16) per step
        int it = 0;
        for (; it < nk; ++it) {
            const int s = it % stages;
            if (!mbar_wait(full + s, (it / stages) & 1)) {
                atomicOr(&s_err, 4u);
                break;
            }
            tc_fence_after();
            unsigned char *st = dsm + (size_t)s * stage_bytes;
            const uint32_t abase = smem_u32(st + (size_t)nl * kXTile);
            for (int q = 0; q < nl; ++q) {
                const uint32_t xbase = smem_u32(st + (size_t)q * kXTile);
#pragma unroll
                for (int kk = 0; kk < kRB / 32; ++kk) {
                    // accumulator of part q: forward, one per limb; backward, hi
                    // in the first and mid + lo in the second (or all three in one)
                    const int qa = kBwd ? (kBwdAcc == 1 ? 0 : (q > 1 ? 1 : q)) : q;
                    const bool first = it == 0 && kk == 0 && (!kBwd || q < kBwdAcc);
                    umma<kN, kF8>(tmem + (uint32_t)(qa * kN), sw_desc<kRB>(xbase + kk * 32), sw_desc<kRB>(abase + kk * 32),
                                  first ? 0u : 1u);
                }
            }
            umma_commit(empty + s);  // frees the stage once these MMAs have read it
        }
        umma_commit(done);  // arrives when every MMA issued above has completed
    }
    __syncwarp();

    // epilogue: every thread owns one source (TMEM lane = 32 * warp + lane);
    // the first 16 columns' frontier words (and sigma values) are fetched
    // while the MMAs run, and each chunk fetches the next one's before its own
    // arithmetic
    const int b = tid & 127;
    const size_t nW = (size_t)p.n * kDW;
    const uint32_t *Fl = Fb + (size_t)l * nW;
    const uint32_t *Vin = Vb + (size_t)(l & 1) * nW;
    uint32_t fw[16];
    uint64_t sv[16];
    epi_prefetch<kBwd>(p.n, Fl, Vin, sigma, v0 + cbeg, warp, b, fw, sv);
    // `good` is uniform across the block (the warp collectives below rely on it)
    const bool ok = mbar_wait(done, 0);
    tc_fence_after();
    const bool good = __syncthreads_and(ok) != 0 && s_err == 0u;
    if (!good && tid == 0) atomicOr(&p.ctl->status, BC_STATUS_DENSE_TIMEOUT);
    if constexpr (kBwd) {
        // per column, the batch's delta values summed as unevaluated FP32 pairs
        // (two-sum over the warp's 32 sources, a fixed tree), then the four
        // warps' pairs in FP64, in warp order
        __shared__ float2 s_red[4][kN];
        const bool valid_src = b < nbv;
        const size_t xr = (size_t)bb * p.xrows + xout + b;  // this source's hi row; mid and lo follow at +128, +256
        // summary terms of this thread's pairs (level l, its columns)
        unsigned long long t_hs = 0, t_vs = 0, t_cnt = 0;
        for (int c0 = cbeg; good && c0 < cbeg + kCols; c0 += 16) {
            uint32_t fwn[16];
            uint64_t svn[16];
            epi_prefetch<true>(p.n, Fl, Vin, sigma, v0 + c0 + 16, warp, b, fwn, svn);
            float S[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) S[i] = 0.0f;
            for (int q = 0; q < kBwdAcc; ++q) {  // all parts, or hi then mid + lo
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(q * kN + c0), r);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) S[i] += __uint_as_float(r[i]);
            }
            uint32_t ph[8], pm[8], pl[8];  // the 16 split c values of this row, two bf16 per word
#pragma unroll
            for (int i = 0; i < 8; ++i) ph[i] = pm[i] = pl[i] = 0u;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int v = v0 + c0 + i;
                float d = 0.0f, c = 0.0f;
                if (v < p.n && valid_src && ((fw[i] >> lane) & 1u)) {
                    t_hs += (unsigned long long)sv[i] * (unsigned long long)(v + 1);
                    t_vs += (unsigned long long)(v + 1);
                    ++t_cnt;
                    const float sg = __ull2float_rn(sv[i]);
                    d = sg * S[i];          // delta_s*(v) = sigma_s(v) * sum_w c_s(w)
                    c = (1.0f + d) / sg;    // c_s(v) for the level above
                }
                float hi = d, lo = 0.0f;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const float h2 = __shfl_xor_sync(0xffffffffu, hi, off);
                    const float l2 = __shfl_xor_sync(0xffffffffu, lo, off);
                    two_sum_add(hi, lo, h2);
                    lo += l2;
                }
                if (lane == 0) s_red[warp][c0 + i] = make_float2(hi, lo);
                const __nv_bfloat16 h = __float2bfloat16_rn(c);
                const float r1 = c - __bfloat162float(h);
                const __nv_bfloat16 m = __float2bfloat16_rn(r1);
                const __nv_bfloat16 lw = __float2bfloat16_rn(r1 - __bfloat162float(m));
                const int sh = 16 * (i & 1);
                ph[i >> 1] |= (uint32_t)__bfloat16_as_ushort(h) << sh;
                pm[i >> 1] |= (uint32_t)__bfloat16_as_ushort(m) << sh;
                pl[i >> 1] |= (uint32_t)__bfloat16_as_ushort(lw) << sh;
            }
            if (write_next) {
                // 32 contiguous bytes per part (npad is a multiple of 128 and
                // c0 of 16, so each store is 16-byte aligned); columns past n
                // get zeros
                uint4 *dh = reinterpret_cast<uint4 *>(p.X + xr * p.npad + v0 + c0);
                uint4 *dm = reinterpret_cast<uint4 *>(p.X + (xr + kDB) * p.npad + v0 + c0);
                uint4 *dl = reinterpret_cast<uint4 *>(p.X + (xr + 2 * kDB) * p.npad + v0 + c0);
                dh[0] = make_uint4(ph[0], ph[1], ph[2], ph[3]);
                dh[1] = make_uint4(ph[4], ph[5], ph[6], ph[7]);
                dm[0] = make_uint4(pm[0], pm[1], pm[2], pm[3]);
                dm[1] = make_uint4(pm[4], pm[5], pm[6], pm[7]);
                dl[0] = make_uint4(pl[0], pl[1], pl[2], pl[3]);
                dl[1] = make_uint4(pl[4], pl[5], pl[6], pl[7]);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                fw[i] = fwn[i];
                sv[i] = svn[i];
            }
        }
        if (good && p.h_sigma && t_cnt) {  // d = l for every pair here
            const size_t o = (size_t)p.src_base + (size_t)bb * kDB + b;
            atomicAdd(reinterpret_cast<unsigned long long *>(p.h_sigma + o), t_hs);
            atomicAdd(reinterpret_cast<unsigned long long *>(p.h_dist + o), (unsigned long long)(l + 1) * t_vs);
            atomicAdd(reinterpret_cast<unsigned long long *>(p.dist_sum + o), (unsigned long long)l * t_cnt);
            atomicAdd(reinterpret_cast<unsigned long long *>(p.reach + o), t_cnt);
        }
        __syncthreads();
        for (int c = tid; good && c < kN && v0 + c < p.n; c += kT) {
            double acc = 0.0;
#pragma unroll
            for (int w = 0; w < 4; ++w) acc += (double)s_red[w][c].x + (double)s_red[w][c].y;
            p.bcpart[(size_t)bb * p.n + v0 + c] += acc;
        }
    } else {
        // the tile's new frontier and visited words, written after the last
        // chunk as one 16-byte row per vertex (and one union word per 32)
        __shared__ uint32_t s_Fw[kN][kDW], s_Vw[kN][kDW];
        uint32_t *Fn = Fb + (size_t)(l + 1) * nW;
        uint32_t *Vout = Vb + (size_t)((l + 1) & 1) * nW;
        uint32_t *ufn = ufb + (size_t)(l + 1) * p.nw32;
        const bool valid_src = b < nbv;
        bool ovf = false, produced = false;
        unsigned long long maxsig = 0, remaining = 0;
        for (int c0 = cbeg; good && c0 < cbeg + kCols; c0 += 16) {
            uint32_t fwn[16];
            uint64_t svn[16];
            epi_prefetch<false>(p.n, Fl, Vin, sigma, v0 + c0 + 16, warp, b, fwn, svn);
            uint64_t lo[16];
            uint32_t hi[16];
    #pragma unroll
            for (int i = 0; i < 16; ++i) {
                lo[i] = 0ull;
                hi[i] = 0u;
            }
            for (int q = 0; q < nl; ++q) {
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(q * kN + c0), r);
                tmem_wait_ld();
    #pragma unroll
                for (int i = 0; i < 16; ++i) {
                    // exact integer < 2^24 held in FP32; add 2^(8q) * a into (hi:lo)
                    const uint64_t a = (uint64_t)__float2uint_rn(__uint_as_float(r[i]));
                    const int sh = (kF8 ? 4 : 8) * q;
                    const uint64_t part = a << sh;
                    const uint64_t carry_bits = sh ? (a >> (64 - sh)) : 0ull;
                    const uint64_t y = lo[i] + part;
                    hi[i] += (uint32_t)carry_bits + (y < part ? 1u : 0u);
                    lo[i] = y;
                }
            }
    #pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int v = v0 + c0 + i;
                if (v >= p.n) continue;  // padding columns (uniform across the block)
                const uint32_t vis = fw[i];
                const bool seen = (vis >> lane) & 1u;
                const bool hit = valid_src && !seen && (lo[i] | hi[i]) != 0ull;
                if (hit) {
                    sigma[(size_t)v * kDB + b] = lo[i];
                    ovf |= hi[i] != 0u;
                    maxsig = lo[i] > maxsig ? lo[i] : maxsig;
                }
                remaining += (valid_src && !seen && !hit) ? 1ull : 0ull;
                const uint32_t word = __ballot_sync(0xffffffffu, hit);
                if (lane == 0) {
                    s_Fw[c0 + i][warp] = word;
                    s_Vw[c0 + i][warp] = vis;
                }
                produced |= word != 0u;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) fw[i] = fwn[i];
        }
        __syncthreads();
        for (int c = tid; good && c < kN; c += kT) {  // kN is a multiple of 32: whole warps per pass
            const int v = v0 + c;
            bool joined = false;
            if (v < p.n) {
                const uint4 f4 = make_uint4(s_Fw[c][0], s_Fw[c][1], s_Fw[c][2], s_Fw[c][3]);
                *reinterpret_cast<uint4 *>(Fn + (size_t)v * kDW) = f4;
                *reinterpret_cast<uint4 *>(Vout + (size_t)v * kDW) =
                    make_uint4(s_Vw[c][0], s_Vw[c][1], s_Vw[c][2], s_Vw[c][3]);
                joined = (f4.x | f4.y | f4.z | f4.w) != 0u;
            }
            const uint32_t bits = __ballot_sync(0xffffffffu, joined);
            if (lane == 0 && bits) atomicOr(ufn + (v >> 5), bits);
        }
        if (good) {
            if (__any_sync(0xffffffffu, ovf) && lane == 0) atomicOr(&p.ctl->status, BC_STATUS_SIGMA_OVERFLOW);
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, maxsig, off);
                maxsig = o > maxsig ? o : maxsig;
                remaining += __shfl_xor_sync(0xffffffffu, remaining, off);
            }
            if (lane == 0) {
                DenseCtl *dc = p.dctl + bb;
                if (produced) atomicOr(&dc->produced, 1u);
                if (maxsig) atomicMax(&dc->maxsig, maxsig);
                if (remaining) atomicAdd(&dc->remaining, remaining);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// Limb matrix of level l: X[q*128 + b][u] = byte q of sigma_b(u) where
// d(s_b, u) = l, else 0 (bf16). Tiles of 32 vertices x 128 sources through
// shared memory so both the sigma reads and the X writes are coalesced. The
// grid covers all npad columns: the padding is written with zeros, since the
// buffer holds other rows' values there (0 x NaN is NaN in the products).
__global__ void __launch_bounds__(256) k_dense_limbs(const DenseParams p, const int l, const int nl) {
    __shared__ uint64_t tile[32][kDB + 1];
    const int u0 = blockIdx.x * 32;
    const int bb = p.blist[blockIdx.y];
    const uint64_t *sigma = p.sigma + (size_t)bb * p.sig_stride;
    __nv_bfloat16 *X = p.X + (size_t)bb * p.xrows * p.npad;
    const size_t nW = (size_t)p.n * kDW;
    const uint32_t *Fl = p.F + (size_t)bb * p.f_stride + (size_t)l * nW;
    for (int i = threadIdx.x; i < 32 * kDB; i += 256) {
        const int uu = i / kDB, b = i % kDB;
        const int u = u0 + uu;
        uint64_t s = 0;
        if (u < p.n && ((__ldg(Fl + (size_t)u * kDW + (b >> 5)) >> (b & 31)) & 1u)) s = sigma[(size_t)u * kDB + b];
        tile[uu][b] = s;
    }
    __syncthreads();
    for (int q = 0; q < nl; ++q) {
        for (int i = threadIdx.x; i < 32 * kDB; i += 256) {
            const int b = i / 32, uu = i % 32;
            const unsigned byte = (unsigned)((tile[uu][b] >> (8 * q)) & 0xFFu);
            X[((size_t)q * kDB + b) * p.npad + u0 + uu] = __float2bfloat16_rn((float)byte);
        }
    }
}

// The same for e4m3 operands: X8[q*128 + b][u] = nibble q (4 bits) of
// sigma_b(u) where d(s_b, u) = l, else 0; every value 0..15 is exact in e4m3.
// Rows of npad bytes; batch b's rows start at b * 2 * xrows. Here too every
// column up to npad is written: the bytes there may belong to bf16 rows of an
// earlier sweep and read as e4m3 NaN. Tiles of 64 vertices x 128 sources
// (counts below 2^16 on this path, kept as 32-bit words); four columns per
// 4-byte store. ones: every count of the level is 1 (level 1, set by
// k_dense_first), so sigma is not read.
__global__ void __launch_bounds__(256) k_dense_nibbles(const DenseParams p, const int l, const int nq,
                                                       const int ones) {
    __shared__ uint32_t tile[64][kDB + 1];
    const int u0 = blockIdx.x * 64;
    const int bb = p.blist[blockIdx.y];
    const uint64_t *sigma = p.sigma + (size_t)bb * p.sig_stride;
    uint8_t *X8 = reinterpret_cast<uint8_t *>(p.X) + (size_t)bb * 2 * p.xrows * p.npad;
    const size_t nW = (size_t)p.n * kDW;
    const uint32_t *Fl = p.F + (size_t)bb * p.f_stride + (size_t)l * nW;
    for (int i = threadIdx.x; i < 64 * kDB; i += 256) {
        const int uu = i / kDB, b = i % kDB;
        const int u = u0 + uu;
        uint32_t s = 0;
        if (u < p.n && ((__ldg(Fl + (size_t)u * kDW + (b >> 5)) >> (b & 31)) & 1u))
            s = ones ? 1u : (uint32_t)sigma[(size_t)u * kDB + b];
        tile[uu][b] = s;
    }
    __syncthreads();
    for (int q = 0; q < nq; ++q) {
        for (int i = threadIdx.x; i < kDB * 16; i += 256) {
            const int b = i / 16, c4 = 4 * (i % 16);
            uint32_t w = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const unsigned nib = (tile[c4 + k][b] >> (4 * q)) & 0xFu;
                w |= (uint32_t)__nv_cvt_float_to_fp8((float)nib, __NV_SATFINITE, __NV_E4M3) << (8 * k);
            }
            *reinterpret_cast<uint32_t *>(X8 + ((size_t)q * kDB + b) * p.npad + u0 + c4) = w;
        }
    }
}

// Split masked c rows of the deepest level L (c_s(v) = 1 / sigma_s(v) there:
// nothing depends on the farthest vertices, Lemma 3.3): rows q*128 + b of the
// batch's first block hold part q (hi, mid, lo) of c, 0 for the pairs not at
// level L. Tiles of 64 vertices x 128 sources through shared memory: sigma is
// read along the sources, the X rows are written along the vertices (two
// columns per 4-byte store); columns past n get zeros.
__global__ void __launch_bounds__(256) k_dense_bwd_last(const DenseParams p) {
    __shared__ float tile[64][kDB + 1];
    const int v0 = blockIdx.x * 64;
    const int bb = blockIdx.y;
    const int L = p.depth[bb];
    const int nbv = p.nbs[bb];
    if (L < 1) {  // no source of the batch has a neighbour: only their own summary terms
        if (p.h_sigma && blockIdx.x == 0 && threadIdx.x < nbv) {
            const size_t o = (size_t)p.src_base + (size_t)bb * kDB + threadIdx.x;
            const unsigned long long h0 = (unsigned long long)p.sources[(size_t)bb * kDB + threadIdx.x] + 1ull;
            atomicAdd(reinterpret_cast<unsigned long long *>(p.h_sigma + o), h0);
            atomicAdd(reinterpret_cast<unsigned long long *>(p.h_dist + o), h0);
            atomicAdd(reinterpret_cast<unsigned long long *>(p.reach + o), 1ull);
        }
        return;
    }
    const size_t nW = (size_t)p.n * kDW;
    const uint32_t *FL = p.F + (size_t)bb * p.f_stride + (size_t)L * nW;
    const uint64_t *sigma = p.sigma + (size_t)bb * p.sig_stride;
    const int bt = threadIdx.x % kDB;  // the source of every item of this thread
    unsigned long long t_hs = 0, t_vs = 0, t_cnt = 0;
    for (int i = threadIdx.x; i < 64 * kDB; i += 256) {
        const int vv = i / kDB, b = i % kDB;
        const int v = v0 + vv;
        float c = 0.0f;
        if (v < p.n && b < nbv && ((__ldg(FL + (size_t)v * kDW + (b >> 5)) >> (b & 31)) & 1u)) {
            const uint64_t sg = sigma[(size_t)v * kDB + b];
            c = 1.0f / __ull2float_rn(sg);
            t_hs += (unsigned long long)sg * (unsigned long long)(v + 1);
            t_vs += (unsigned long long)(v + 1);
            ++t_cnt;
        }
        tile[vv][b] = c;
    }
    if (p.h_sigma) {
        // summaries: this thread's level-L pairs, and (first tile) the source
        // itself, d = 0 and sigma = 1
        unsigned long long h0 = 0, c0 = 0;
        if (blockIdx.x == 0 && threadIdx.x < kDB && bt < nbv) {
            h0 = (unsigned long long)p.sources[(size_t)bb * kDB + bt] + 1ull;
            c0 = 1;
        }
        if (t_cnt || c0) {
            const size_t o = (size_t)p.src_base + (size_t)bb * kDB + bt;
            atomicAdd(reinterpret_cast<unsigned long long *>(p.h_sigma + o), t_hs + h0);
            atomicAdd(reinterpret_cast<unsigned long long *>(p.h_dist + o), (unsigned long long)(L + 1) * t_vs + h0);
            atomicAdd(reinterpret_cast<unsigned long long *>(p.dist_sum + o), (unsigned long long)L * t_cnt);
            atomicAdd(reinterpret_cast<unsigned long long *>(p.reach + o), t_cnt + c0);
        }
    }
    __syncthreads();
    __nv_bfloat16 *X = p.X + (size_t)bb * p.xrows * p.npad;  // block 0 holds level L
    for (int i = threadIdx.x; i < kDB * 32; i += 256) {
        const int b = i / 32, vv = 2 * (i % 32);
        uint32_t w[3] = {0u, 0u, 0u};
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float c = tile[vv + k][b];
            const __nv_bfloat16 h = __float2bfloat16_rn(c);
            const float r1 = c - __bfloat162float(h);
            const __nv_bfloat16 m = __float2bfloat16_rn(r1);
            const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(m));
            w[0] |= (uint32_t)__bfloat16_as_ushort(h) << (16 * k);
            w[1] |= (uint32_t)__bfloat16_as_ushort(m) << (16 * k);
            w[2] |= (uint32_t)__bfloat16_as_ushort(lo) << (16 * k);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q)
            *reinterpret_cast<uint32_t *>(X + ((size_t)q * kDB + b) * p.npad + v0 + vv) = w[q];
    }
}

// Levels 0 and 1 of every batch of a group in one launch (blockIdx.y = batch):
// d(s,s) = 0 and sigma_s(s) = 1, and each neighbour v of s has d(s,v) = 1 and
// sigma_s(v) = 1, its one shortest path being the arc s-v (the CSR holds no
// duplicate arcs and no self-loops; Section 1.1). The group's frontier words
// of levels 0 and 1, its visited words and its union-frontier bits are zero
// when the launch starts. One warp per source, its lanes over the arcs.
__global__ void __launch_bounds__(256) k_dense_first(const DenseParams p, const int32_t *__restrict__ sources,
                                                     const int32_t *__restrict__ row_ptr,
                                                     const int32_t *__restrict__ col) {
    const int bb = blockIdx.y;
    const int nbv = p.nbs[bb];
    const size_t nW = (size_t)p.n * kDW;
    uint32_t *F = p.F + (size_t)bb * p.f_stride;
    uint32_t *V = p.V + (size_t)bb * p.v_stride;
    uint32_t *uf = p.ufr + (size_t)bb * p.u_stride;
    uint64_t *sigma = p.sigma + (size_t)bb * p.sig_stride;
    const int32_t *src = sources + (size_t)bb * kDB;
    const int lane = threadIdx.x & 31;
    for (int b = blockIdx.x * 8 + (threadIdx.x >> 5); b < nbv; b += gridDim.x * 8) {
        const int s = src[b];
        const uint32_t bit = 1u << (b & 31);
        if (lane == 0) {
            atomicOr(F + (size_t)s * kDW + (b >> 5), bit);           // frontier 0
            atomicOr(V + nW + (size_t)s * kDW + (b >> 5), bit);      // visited through level 0
            atomicOr(uf + (s >> 5), 1u << (s & 31));
            sigma[(size_t)s * kDB + b] = 1ull;
        }
        for (int e = row_ptr[s] + lane; e < row_ptr[s + 1]; e += 32) {
            const int v = col[e];
            atomicOr(F + nW + (size_t)v * kDW + (b >> 5), bit);      // frontier 1
            atomicOr(uf + p.nw32 + (v >> 5), 1u << (v & 31));
            sigma[(size_t)v * kDB + b] = 1ull;
        }
    }
}

// BC of a group: bc[v] += sum_b bcpart[b][v], batches in order.
__global__ void __launch_bounds__(256) k_dense_bc_reduce(const double *__restrict__ part, int nbatch, int n,
                                                         double *__restrict__ bc) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int b = 0; b < nbatch; ++b) acc += part[(size_t)b * n + v];
        bc[v] += acc;
    }
}

// Dense 0/1 adjacency in bf16 from the CSR (rows beyond n and columns beyond
// n stay zero).
__global__ void k_dense_adjacency(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int32_t n,
                                  int32_t npad, __nv_bfloat16 *A) {
    for (int v = blockIdx.x; v < n; v += gridDim.x)
        for (int e = row_ptr[v] + threadIdx.x; e < row_ptr[v + 1]; e += blockDim.x)
            A[(size_t)v * npad + col[e]] = __float2bfloat16_rn(1.0f);
}

// The same adjacency in e4m3 (1.0 = 0x38, 0 = 0x00), one byte per entry.
__global__ void k_dense_adjacency8(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int32_t n,
                                   int32_t npad, uint8_t *A8) {
    const uint8_t one = (uint8_t)__nv_cvt_float_to_fp8(1.0f, __NV_SATFINITE, __NV_E4M3);
    for (int v = blockIdx.x; v < n; v += gridDim.x)
        for (int e = row_ptr[v] + threadIdx.x; e < row_ptr[v + 1]; e += blockDim.x) A8[(size_t)v * npad + col[e]] = one;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

// Boxes of kK elements (the swizzle span: 128 or 64 bytes) by box_rows rows;
// bf16 elements, or bytes (e4m3) when f8.
bool make_map(CUtensorMap *m, void *base, uint64_t inner, uint64_t rows, uint32_t box_rows, int kK, bool f8 = false) {
    auto fn = encode_fn();
    if (!fn) return false;
    const uint64_t esz = f8 ? 1 : 2;
    const cuuint64_t dims[2] = {inner, rows};
    const cuuint64_t strides[1] = {inner * esz};
    const cuuint32_t box[2] = {(cuuint32_t)kK, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              kK * esz == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

template <int kN, int kK, bool kF8 = false>
int dense_stages(int nl, bool bwd = false) {
    // accumulators of at most 128 TMEM columns: three CTAs per SM, at most
    // 256: two (so one CTA's epilogue overlaps the others' MMAs), more: one
    // CTA with most of the shared memory in stages
    const int nacc = bwd ? kBwdAcc : nl;
    const int budget = nacc * kN <= 128 ? 66 * 1024 : (nacc * kN <= 256 ? 100 * 1024 : 200 * 1024);
    const int s = budget / (nl * x_tile<kK, kF8>() + a_tile<kN, kK, kF8>());
    return s < 1 ? 1 : (s > 8 ? 8 : s);
}

template <int kN, int kK, bool kF8 = false>
size_t dense_smem_bytes(int nl, int stages) {
    return (size_t)stages * (nl * x_tile<kK, kF8>() + a_tile<kN, kK, kF8>()) + 1024 + (2 * stages + 2) * sizeof(uint64_t) +
           64;
}

int dense_build_adjacency(const int32_t *row_ptr, const int32_t *col, int32_t n, int32_t npad, __nv_bfloat16 *A,
                          cudaStream_t st) {
    if (cudaMemsetAsync(A, 0, (size_t)npad * npad * sizeof(__nv_bfloat16), st) != cudaSuccess) return -1;
    if (n > 0) k_dense_adjacency<<<n < 4096 ? n : 4096, 128, 0, st>>>(row_ptr, col, n, npad, A);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int dense_build_adjacency8(const int32_t *row_ptr, const int32_t *col, int32_t n, int32_t npad, uint8_t *A8,
                           cudaStream_t st) {
    if (cudaMemsetAsync(A8, 0, (size_t)npad * npad, st) != cudaSuccess) return -1;
    if (n > 0) k_dense_adjacency8<<<n < 4096 ? n : 4096, 128, 0, st>>>(row_ptr, col, n, npad, A8);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int dense_make_maps(DenseMaps *maps, __nv_bfloat16 *X, uint64_t xrows_total, __nv_bfloat16 *A, uint8_t *A8,
                    int32_t npad) {
    maps->has_f8 = false;
    if (A8) {  // e4m3 operands: X rows of npad bytes (two per bf16 row), adjacency boxes of 128 rows
        if (!make_map(&maps->x8, X, (uint64_t)npad, 2 * xrows_total, kDB, 128, true)) return -1;
        if (!make_map(&maps->a8, A8, (uint64_t)npad, (uint64_t)npad, kNW, 128, true)) return -1;
        maps->has_f8 = true;
    }
    if (!make_map(&maps->x, X, (uint64_t)npad, xrows_total, kDB, 64)) return -1;
    if (!make_map(&maps->a, A, (uint64_t)npad, (uint64_t)npad, kNT, 64)) return -1;
    if (!make_map(&maps->a_wide, A, (uint64_t)npad, (uint64_t)npad, kNW, 64)) return -1;
    if (!make_map(&maps->x32, X, (uint64_t)npad, xrows_total, kDB, 32)) return -1;
    if (!make_map(&maps->a_wide32, A, (uint64_t)npad, (uint64_t)npad, kNW, 32)) return -1;
    if (npad % kNX == 0) {
        if (!make_map(&maps->a_x, A, (uint64_t)npad, (uint64_t)npad, kNX, 64)) return -1;
        if (!make_map(&maps->a_x32, A, (uint64_t)npad, (uint64_t)npad, kNX, 32)) return -1;
    }
    return 0;
}

// Stage K (elements) of the bf16 forward and backward level kernels.
constexpr int kFwdK = 64;
constexpr int kBwdK = 32;
// Backward tiles of 256 vertices when npad allows: its two accumulators fill
// TMEM (one CTA per SM, five K = 32 stages), and the CTA's 8 warps split the
// epilogue's columns in two.
constexpr bool kBwdX = true;
constexpr int kBwdXThreads = 256;
// The forward's limb products in e4m3 with 4-bit limbs (kind::f8f6f4: one
// byte per operand element and twice the bf16 rate) while the level's counts
// need at most four of them (below 2^16); bf16 8-bit limbs otherwise.
constexpr bool kFwdF8 = true;
// A bf16 one-limb forward on 256-vertex tiles (kFwdXK elements per stage)
// measured the same as on 128, so it is off.
constexpr bool kFwdX = false;
constexpr int kFwdXK = 64;

// A CTA covers kNW = 128 vertices when the limb accumulators fit TMEM
// (nl * 128 <= 512 columns), else kNT = 64.
template <bool kBwd, int kN, int kK, bool kF8 = false>
int launch_level_t(const DenseMaps &maps, const DenseParams &p, int l, int nl, int write_next, cudaStream_t st) {
    const int stages = dense_stages<kN, kK, kF8>(nl, kBwd);
    const size_t smem = dense_smem_bytes<kN, kK, kF8>(nl, stages);
    // the widest backward tile runs one CTA per SM: its epilogue gets 8 warps
    constexpr int kT = (kBwd && kN == kNX) ? kBwdXThreads : 128;
    if (cudaFuncSetAttribute(k_dense_level<kBwd, kN, kK, kT, kF8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return -1;
    const CUtensorMap &mx = kF8 ? maps.x8 : (kK == 64 ? maps.x : maps.x32);
    const CUtensorMap &ma = kF8 ? maps.a8
                                : (kN == kNX ? (kK == 64 ? maps.a_x : maps.a_x32)
                                             : (kK == 64 ? (kN == kNW ? maps.a_wide : maps.a) : maps.a_wide32));
    k_dense_level<kBwd, kN, kK, kT, kF8><<<p.nactive * (p.npad / kN), kT, smem, st>>>(mx, ma, p, l, nl, stages,
                                                                                       write_next);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

bool dense_level_f8(const DenseMaps &maps, int nq) { return kFwdF8 && maps.has_f8 && nq >= 1 && nq <= 4; }

int dense_launch_level(const DenseMaps &maps, const DenseParams &p, int l, int nl, int nq, cudaStream_t st) {
    if (p.nactive <= 0) return 0;
    if (dense_level_f8(maps, nq)) {  // 4-bit limbs in e4m3, 128-vertex tiles
        k_dense_nibbles<<<dim3(p.npad / 64, p.nactive), 256, 0, st>>>(p, l, nq, l == 1 ? 1 : 0);
        return launch_level_t<false, kNW, 128, true>(maps, p, l, nq, 0, st);
    }
    k_dense_limbs<<<dim3(p.npad / 32, p.nactive), 256, 0, st>>>(p, l, nl);
    if (kFwdX && nl == 1 && p.npad % kNX == 0) return launch_level_t<false, kNX, kFwdXK>(maps, p, l, nl, 0, st);
    if (nl * kNW <= 512) return launch_level_t<false, kNW, kFwdK>(maps, p, l, nl, 0, st);
    return launch_level_t<false, kNT, 64>(maps, p, l, nl, 0, st);
}

int dense_launch_first(const DenseParams &p, int nbatch, const int32_t *sources, const int32_t *row_ptr,
                       const int32_t *col, cudaStream_t st) {
    if (nbatch <= 0 || p.n <= 0) return 0;
    // the group's level-0/1 frontier words, visited words and union bits start at zero
    if (cudaMemset2DAsync(p.F, p.f_stride * sizeof(uint32_t), 0, (size_t)2 * p.n * kDW * sizeof(uint32_t), nbatch,
                          st) != cudaSuccess)
        return -1;
    if (cudaMemsetAsync(p.V, 0, (size_t)nbatch * p.v_stride * sizeof(uint32_t), st) != cudaSuccess) return -1;
    if (cudaMemsetAsync(p.ufr, 0, (size_t)nbatch * p.u_stride * sizeof(uint32_t), st) != cudaSuccess) return -1;
    k_dense_first<<<dim3(kDB / 8, nbatch), 256, 0, st>>>(p, sources, row_ptr, col);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int dense_launch_bwd_last(const DenseParams &p, int nbatch, cudaStream_t st) {
    if (nbatch <= 0 || p.n <= 0) return 0;
    k_dense_bwd_last<<<dim3((p.n + 63) / 64, nbatch), 256, 0, st>>>(p);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int dense_launch_bwd_level(const DenseMaps &maps, const DenseParams &p, int l, cudaStream_t st) {
    if (p.nactive <= 0) return 0;
    if (kBwdX && p.npad % kNX == 0)
        return launch_level_t<true, kNX, kBwdK>(maps, p, l, 3, l > 1 ? 1 : 0, st);  // hi, mid, lo parts
    return launch_level_t<true, kNW, kBwdK>(maps, p, l, 3, l > 1 ? 1 : 0, st);
}

int dense_reduce_bc(const double *bcpart, int nbatch, int n, double *bc, cudaStream_t st) {
    if (n <= 0 || nbatch <= 0) return 0;
    const int g = (n + 255) / 256;
    k_dense_bc_reduce<<<g < 1024 ? g : 1024, 256, 0, st>>>(bcpart, nbatch, n, bc);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace bcgb
