// tc_field.cu -- stale dipole field of a window for all replicas on the
// 5th-generation tensor cores (tcgen05), in split-BF16x3 with FP32 accumulation.
//
// For the S_w sites of a window (Sec. 3.1 update sites of B consecutive
// sub-steps) and every replica r:
//     H0[r][b*S_w + s] = sum_{a, m} W~_{ba}(q_s - m) s_r^a(m)          (Sec. 2.1, Eq. 2)
// is a GEMM D[M x N] = A[M x K] B[K x N] with
//     rows M  = (b, s): in-plane rows b in {x, y} contract over K = (a in {x, y}, m),
//                       zz rows contract over K = (z, m)  (the tensor is block diagonal),
//     cols N  = replicas,
//     A       = the Toeplitz tile W~(q_s - m), built in shared memory from the
//               L^2-entry tensor (8 pre-shifted bf16 copies so that every 16-byte
//               chunk is an aligned vector load),
//     B       = the spins of the replicas, bf16 hi/lo, row r = [x-plane | y-plane | z-plane].
// Each value v is split v = hi + lo (hi = bf16(v), lo = bf16(v - hi)) and the
// product is hi_A hi_B + hi_A lo_B + lo_A hi_B (off by at most ~3 x 2^-16 relative).
//
// One CTA = one (M-tile of 128 rows, N-tile of up to 256 replicas, range of
// K-blocks of 32).  Operands sit in the canonical K-major, no-swizzle
// core-matrix layout (8 rows x 16 bytes per core matrix) in a ring of 4 stages
// handed between warp roles through mbarriers (no CTA-wide barrier in the K
// loop): four producer warps gather the Toeplitz A tile with cp.async, one
// thread per row; one thread loads the spin tile B by TMA, one 2D box of 8
// K-elements x NT replicas per core-matrix column (rows past R arrive as
// zeros); one thread issues tcgen05.mma (M=128, N=tile, K=16) into a TMEM
// accumulator as soon as a stage's operands have landed and commits the stage
// back to the producers.  The epilogue reads TMEM with tcgen05.ld and stores the
// unit's partial tile (split-K); the sub-step kernel sums the partial tiles of
// each output tile in a fixed order as it loads the window (deterministic, no
// atomics).
#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "internal.cuh"
#include "tc_field.cuh"

namespace dipmc {

namespace {

constexpr int kTcThreads = 256;              // two threads per row of the 128-row tile
constexpr int kKB = 32;                       // K elements per stage
constexpr int kKC = kKB / 8;                  // core matrices along K per row
constexpr int kSBO = kKC * 128;               // bytes between 8-row groups
constexpr int kTileA = 128 * kKB * 2;         // bytes of one A tile (hi or lo)
constexpr int kMaxNT = 256;
constexpr int kTileB = kMaxNT * kKB * 2;      // bytes of one B tile (hi or lo)
constexpr int kStage = 2 * kTileA + 2 * kTileB;
constexpr int kStages = 4;
constexpr long long kWaitCycles = 4LL << 30;  // bounded mbarrier waits (~2 s at 2 GHz)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Canonical no-swizzle K-major layout: element (row, k) of a tile with kKB K
// columns lives at (row/8)*kSBO + (k/8)*128 + (row%8)*16 + (k%8)*2 bytes:
// core matrices of 8 rows x 8 elements (128 B); adjacent along K: 128 B
// (leading byte offset), adjacent along M/N: kSBO bytes (stride byte offset).
__device__ __forceinline__ uint32_t core_off(int row, int kc) { return (row >> 3) * kSBO + kc * 128 + (row & 7) * 16; }

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo = 128u, uint32_t sbo = (uint32_t)kSBO) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);          // start address
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;      // leading byte offset (K direction)
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;      // stride byte offset (M/N direction)
    d |= (uint64_t)1 << 46;                           // descriptor version for tcgen05
    // base offset 0, layout type 0 = no swizzle
    return d;
}

// B tile as the TMA boxes leave it: core-matrix column kc (8 K-elements of all
// NT rows) at kc * NT * 16 bytes, 8-row groups 128 bytes apart.
// B tiles (NT rows of kKB = 32 bf16 = 64 bytes, K-major) in the 64-byte swizzled layout
// that the TMA writes with CU_TENSOR_MAP_SWIZZLE_64B: 8-row groups of 512 bytes, the
// 16-byte chunk index of a row XORed with (row / 2) % 4.  The descriptor's start address
// steps by 32 bytes per 16-element K slice; the tile base is 512-byte aligned.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);          // start address
    d |= (uint64_t)1 << 16;                           // leading byte offset (unused when swizzled)
    d |= (uint64_t)(512u >> 4) << 32;                 // stride byte offset: 8 rows x 64 bytes
    d |= (uint64_t)1 << 46;                           // descriptor version for tcgen05
    d |= (uint64_t)4 << 61;                           // layout: 64-byte swizzle
    return d;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}

// 2D TMA load of a box at (x, y) of the tensor map into shared memory.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint64_t *m) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(m))
        : "memory");
}

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
    return (1u << 4)                  // D format: F32
           | (1u << 7)                // A format: BF16
           | (1u << 10)               // B format: BF16
           | ((uint32_t)(N >> 3) << 17)
           | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; returns false (and leaves the error flag to the caller) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *m, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(m, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

// 16-byte asynchronous global -> shared copy (L2 only); src_bytes = 0 fills zeros.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}


__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *m) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(m))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Arrive on m once every cp.async this thread has issued so far has landed (the
// barrier's count includes these arrivals).
__device__ __forceinline__ void cp_async_arrive(uint64_t *m) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(m)) : "memory");
}

// Bounded wait that gives up early once another role has given up; the first
// role to time out raises the CTA's abort flag.
__device__ __forceinline__ bool mbar_wait_abort(uint64_t *m, uint32_t parity, volatile int *abort) {
    const long long t0 = clock64();
    while (!mbar_try_wait(m, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort = 1;
            return false;
        }
    }
    return true;
}

// Warp roles of a CTA (one unit):
//   warp 0, lane 0  issues the MMAs of each stage once its A rows and B tile have
//                   landed, and commits the stage's slot back to the producers;
//   warp 1, lane 0  loads the spin tile B of each stage by TMA;
//   warps 4..7      gather the Toeplitz tile A, one thread per tile row; each
//                   thread's arrival on the stage's barrier fires when its copies
//                   have landed;
//   all warps       read the accumulator out of TMEM at the end.
// No CTA-wide barrier in the K loop: the ring of kStages slots is handed between
// the roles through mbarriers.
constexpr int kProdWarp0 = 4;
constexpr int kProducers = kTcThreads - kProdWarp0 * 32;   // 128: one per tile row
static_assert(kProducers == 128, "one producer per tile row");

__global__ void __launch_bounds__(kTcThreads, 1) k_tc_field(const TcFieldArgs a, const __grid_constant__ CUtensorMap tm_hi,
                                                           const __grid_constant__ CUtensorMap tm_lo) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t afull[kStages];      // the A rows of a stage landed (one arrival per producer)
    __shared__ uint64_t bfull[kStages];      // the TMA bytes of a stage's B tile arrived
    __shared__ uint64_t empty[kStages];      // the MMAs that read a stage completed (slot free)
    __shared__ uint64_t done;                // every MMA of the unit completed
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;
    __shared__ int2 s_rinfo[kProducers];     // spectra: per tile row, offset x | y << 16 and kappa | b << 2
    volatile int *abort = &abort_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (smem_u32(smem) & 1023u) {          // the swizzled B tiles need aligned stages
        if (tid == 0) atomicExch(a.error, 2);
        return;
    }

    // ---- this CTA's unit: M-tile, N-tile, K-block range
    const TcUnit u = a.units[blockIdx.x];
    const int L = a.L, N = L * L, Sw = a.Sw;
    const int row0 = u.mtile * 128;                 // first row (b*Sw + s) of the tile
    const bool zz = row0 >= 2 * Sw;
    const int n0 = u.ntile * a.NT;                  // first replica of the tile
    const int nrows_b = a.NT;                       // N of the MMA
    const uint32_t idesc = make_idesc(128, nrows_b);
    const int nkb = u.kb_end - u.kb_begin;

    // producer thread: its tile row's window site and tensor components
    const bool producer = warp >= kProdWarp0;
    const int arow = tid - kProdWarp0 * 32;
    int my_b = 0, my_qx = 0, my_qy = 0, my_kap = 0;
    int sp_xy[4] = {0, 0, 0, 0}, sp_kb[4] = {0, 0, 0, 0};   // spectra: rows arow / 4 + 32 m
    if (producer) {
        const int my_row = row0 + arow;
        int slot;                                    // window site (Toeplitz) or first site of the offset (spectra)
        if (a.spec2) {
            // rows kappa*2B + b*B + j (in-plane) and 2 S_w + (kappa/2)*2B + (kappa%2)*B + j (zz), B = S_w/4
            const int B4 = Sw >> 2;
            if (my_row < 2 * Sw) {
                my_kap = my_row / (2 * B4);
                my_b = (my_row / B4) & 1;
            } else {
                const int rz = my_row - 2 * Sw;
                my_kap = 2 * (rz / (2 * B4)) + ((rz / B4) & 1);
                my_b = 2;
            }
            slot = 4 * (my_row % B4);
        } else {
            my_b = my_row / Sw;                      // output component 0 x, 1 y, 2 z
            slot = my_row - my_b * Sw;
        }
        const uint32_t t = a.t_dev ? *a.t_dev + (uint32_t)a.it : a.t_host;
        const uint4 rk = a.schedule == 0 ? philox(make_uint4(t, 0u, 0u, kTagPerm), a.key) : make_uint4(0, 0, 0, 0);
        const int xy = window_site_xy(a.l, L / a.l, a.key, t, a.schedule, rk, a.k0, slot);
        my_qx = xy & 0xFFFF;                         // spectra: the offset (ox, oy) of the row's sub-step
        my_qy = xy >> 16;
        if (a.spec2) {
            // spectra rows are copied four lanes to a row (each lane one 16-byte chunk of the
            // row's 64 bytes, so a warp's copies touch 8 rows instead of 32): lane arow takes
            // rows arow / 4 + 32 m, m = 0..3, at chunk arow % 4
            s_rinfo[arow] = make_int2(xy, my_kap | (my_b << 2));
            asm volatile("bar.sync 1, %0;" ::"n"(kProducers) : "memory");
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int2 ri = s_rinfo[(arow >> 2) + 32 * m];
                sp_xy[m] = ri.x;
                sp_kb[m] = ri.y;
            }
        }
    }
    if (warp == 0) {
        // TMEM accumulator: 128 lanes x NT fp32 columns (allocation is a power of 2 >= 32)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"((uint32_t)a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&afull[s], kProducers);
            mbar_init(&bfull[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_s;
    // Under programmatic dependent launch everything up to here, and the gather of
    // the Toeplitz operand (it reads only W~), overlaps the previous kernel's tail;
    // the spin tiles (B) and the partial-tile stores (the previous window's sub-step
    // kernel reads that buffer) wait for it.

    if (producer) {
        // ---- A: Toeplitz rows W~(q - m) of K-block i into slot i % kStages
        const int comp_a0 = my_b == 0 ? 0 : 1;             // (b, a = x): xx or xy
        const int comp_a1 = my_b == 0 ? 1 : 2;             // (b, a = y): xy or yy
        for (int i = 0; i < nkb; ++i) {
            const int s = i % kStages;
            if (i >= kStages && !mbar_wait_abort(&empty[s], (uint32_t)(((i / kStages) - 1) & 1), abort)) break;
            const uint32_t sAhi = smem_u32(smem + s * kStage), sAlo = sAhi + kTileA;
            const int k0 = (u.kb_begin + i) * kKB;             // K offset within this tile's contraction
            if (a.spec2) {
                // signed spectrum of W~ at (o - e) mod l for the offsets e = e0 .. e0+31 (cell
                // offsets in the order e' = ey*l + (l-1-ex), so each 8-run is ascending in i)
                const int l = a.l, lsq = l * l, l2 = 2 * l;
                const int part = k0 >= lsq;                    // in-plane: input component; zz: kappa of the pair
                const int kc = arow & 3;
                const int e = k0 - part * lsq + 8 * kc, ey = e / l, exq = e - ey * l;
                const size_t cstride = (size_t)4 * 4 * 2 * 2 * l * l2;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int kap = sp_kb[m] & 3, b = sp_kb[m] >> 2;
                    const int comp = b == 2 ? 3 : b + part;   // (b, a): xx, xy | xy, yy; zz
                    const uint32_t bytes = (b == 2 && part != (kap & 1)) ? 0u : 16u;   // zz rows: own kappa only
                    int dy = (sp_xy[m] >> 16) - ey;
                    const int sy = dy < 0;
                    dy += sy ? l : 0;
                    const int i0 = (sp_xy[m] & 0xFFFF) + 1 + exq, c = i0 & 7;
                    const size_t off = (size_t)c * cstride +
                                       ((((size_t)kap * 4 + comp) * 2 + sy) * 2) * l * l2 + (size_t)dy * l2 + (i0 - c);
                    const int ar = (arow >> 2) + 32 * m;
                    cp_async16(sAhi + core_off(ar, kc), a.wsh + off, bytes);
                    cp_async16(sAlo + core_off(ar, kc), a.wsh + off + (size_t)l * l2, bytes);
                }
                cp_async_arrive(&afull[s]);
                continue;
            }
            const int al = zz ? 2 : (k0 >= N ? 1 : 0);         // input component of this K block
            const int comp = zz ? 3 : (al == 0 ? comp_a0 : comp_a1);
            const int m0 = k0 - (zz ? 0 : al * N);             // first source site
            int my = m0 / L, mx = m0 - my * L;
            const __nv_bfloat16 *wc = a.wsh + (size_t)comp * 2 * L * 2 * L;
#pragma unroll
            for (int kc = 0; kc < kKC; ++kc) {
                int dy = my - my_qy;
                if (dy < 0) dy += L;
                int x0 = mx - my_qx;                      // W~(q - m) = W~(m - q): forward segment from x0
                if (x0 < 0) x0 += L;
                const size_t off = (size_t)(x0 & 7) * 4 * 2 * L * 2 * L + (size_t)dy * (2 * L) + (x0 & ~7);
                cp_async16(sAhi + core_off(arow, kc), wc + off, 16);
                cp_async16(sAlo + core_off(arow, kc), wc + off + (size_t)L * 2 * L, 16);
                mx += 8;
                if (mx >= L) { mx -= L; ++my; }
            }
            cp_async_arrive(&afull[s]);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");   // no copy outlives the CTA
    } else if (warp == 1) {
        if (lane == 0) {
            pdl_wait();
            // the next kernel (the sub-step kernel) may launch once every CTA is past this
            // wait: every kernel before this one has then completed, so that kernel may read
            // the spins before its own wait
            pdl_trigger();
            // ---- B: spins of NT replicas x kKB by TMA (x = K offset, a multiple of 8
            // elements = 16 bytes; rows past R read as zeros)
            int issued = 0;
            for (int i = 0; i < nkb; ++i) {
                const int s = i % kStages;
                if (i >= kStages && !mbar_wait_abort(&empty[s], (uint32_t)(((i / kStages) - 1) & 1), abort)) break;
                const int kk = (u.kb_begin + i) * kKB;
                int kofs;
                if (a.spec2) {
                    // spectra [kappa][a][e']: in-plane rows kappa*2B + b*B + j and zz rows
                    // (kappa/2)*2B + (kappa%2)*B + j, B = S_w/4, so a 128-row tile holds one
                    // kappa (in-plane; 2B/128 tiles a kappa) or lies in one kappa pair (zz)
                    const int lsq = N >> 2, B4 = Sw >> 2;
                    if (!zz) {
                        kofs = (u.mtile * 128 / (2 * B4)) * 3 * lsq + kk;
                    } else {
                        const int part = kk >= lsq, pair = (u.mtile - 2 * Sw / 128) * 128 / (2 * B4);
                        kofs = (2 * pair + part) * 3 * lsq + 2 * lsq + (kk - part * lsq);
                    }
                } else {
                    kofs = (zz ? 2 * N : 0) + kk;
                }
                const uint32_t sBhi = smem_u32(smem + s * kStage) + 2 * kTileA, sBlo = sBhi + kTileB;
                mbar_expect_tx(&bfull[s], (uint32_t)(2 * nrows_b * kKB * 2));
                tma_load_2d(sBhi, &tm_hi, kofs, n0, &bfull[s]);   // one 64-byte swizzled box row per replica
                tma_load_2d(sBlo, &tm_lo, kofs, n0, &bfull[s]);
                issued = i + 1;
            }
            // every issued copy lands before the CTA may leave (each slot's latest use)
            for (int i = issued > kStages ? issued - kStages : 0; i < issued; ++i)
                mbar_wait(&bfull[i % kStages], (uint32_t)((i / kStages) & 1));
        }
        __syncwarp();
    } else if (warp == 0) {
        if (lane == 0) {
            // ---- MMAs: stage i once both operands landed; the commit frees the slot
            for (int i = 0; i < nkb; ++i) {
                const int s = i % kStages;
                const uint32_t par = (uint32_t)((i / kStages) & 1);
                if (!mbar_wait_abort(&afull[s], par, abort) || !mbar_wait_abort(&bfull[s], par, abort)) break;
                // the A rows were written by the producers' cp.async (generic proxy); the
                // MMAs read them through the async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ah = smem_u32(smem + s * kStage);
                const uint32_t alo = ah + kTileA, bh = ah + 2 * kTileA, blo = bh + kTileB;
#pragma unroll
                for (int ks = 0; ks < kKB / 16; ++ks) {
                    const uint32_t ko = ks * 256;        // A: 16 K elements = 2 core matrices = 256 B
                    const uint32_t kb = ks * 32;         // B: 16 K elements of a 64-byte swizzled row
                    const uint32_t acc0 = (i > 0 || ks > 0) ? 1u : 0u;
                    umma_bf16(tmem, smem_desc(ah + ko), smem_desc_sw64(bh + kb), idesc, acc0);
                    umma_bf16(tmem, smem_desc(ah + ko), smem_desc_sw64(blo + kb), idesc, 1u);
                    umma_bf16(tmem, smem_desc(alo + ko), smem_desc_sw64(bh + kb), idesc, 1u);
                }
                umma_commit(&empty[s]);
            }
            umma_commit(&done);   // arrives once every MMA issued above has completed
        }
        __syncwarp();
    }
    // ---- all warps: the accumulator is complete (or the unit gave up)
    pdl_wait();
    const bool fin = mbar_wait(&done, 0u);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool ok = fin && !*abort;
    if (!ok) {
        if (tid == 0) atomicExch(a.error, 1);
    } else if (nkb > 0) {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 = rows of the tile,
        // warps w and w + 4 alternate 32-column chunks; the partial tile goes to the
        // unit's slot, row fastest (a warp stores 128 B per column)
        const int wl = warp & 3;
        float *pt = a.part + (size_t)blockIdx.x * nrows_b * 128 + wl * 32 + lane;
        for (int cb = (warp >> 2) * 32; cb < nrows_b; cb += 64) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(wl * 32) << 16) + (uint32_t)cb, v);
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (cb + j < nrows_b) pt[(size_t)(cb + j) * 128] = v[j];   // NT may end mid-chunk (NT % 32 == 16)
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)a.tmem_cols)
                     : "memory");
    }
}

// 8 shifted, doubled bf16 hi/lo copies of W~: wsh[c][comp][hl][y][i] = part_hl(W~_comp(y, (i + c) mod L)),
// i in [0, 2L).  Any 8 consecutive columns starting at x0 are then the aligned
// 16 bytes at i = x0 - (x0 mod 8) of copy c = x0 mod 8.
__global__ void k_build_wsh(int L, const double *__restrict__ W64, __nv_bfloat16 *wsh) {
    const size_t total = (size_t)8 * 4 * L * 2 * L;
    const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    const int i = (int)(gid % (2 * L));
    size_t rest = gid / (2 * L);
    const int y = (int)(rest % L);
    rest /= L;
    const int comp = (int)(rest % 4);
    const int c = (int)(rest / 4);
    const int x = (i + c) % L;
    const int N = L * L;
    const float v = (float)W64[comp * N + y * L + x];
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    const size_t base = (((size_t)c * 4 + comp) * 2) * L * 2 * L;
    wsh[base + (size_t)y * 2 * L + i] = hi;
    wsh[base + (size_t)L * 2 * L + (size_t)y * 2 * L + i] = lo;
}

// Spectral operand mode, L = 2l.  The 2 x 2 cell grid has the real DFT
// F(kappa) = sum_D (-1)^(kappa.D) f(o + l D), kappa = Kx + 2 Ky, D = Dx + 2 Dy (Sec. 3.1
// sub-lattices); the field at o + l D is h = (1/4) sum_kappa (-1)^(kappa.D) H_o(kappa) with
//     H_o(kappa) = sum_e (-1)^(Kx sx + Ky sy) T_{(o - e) mod l}(kappa) S_e(kappa),
// sx, sy = 1 where o - e wraps in x, y, and T, S the DFTs of W~ and of the spins.
// The table holds, for each kappa, component and y-wrap sy, the row
//     T2[dy][i] = (-1)^(Ky sy) (i >= l ? T_(dy, i-l) : (-1)^Kx T_(dy, i)),  i in [0, 2l),
// so that the entries for e' = ey*l + (l-1-ex), ex descending, are T2[dy][ox + 1 + (l-1-ex)]:
// an ascending run; copy c is shifted by c so that every 8-run is one aligned 16 bytes.
__global__ void k_build_t2(int L, const double *__restrict__ W64, __nv_bfloat16 *t2) {
    const int l = L / 2, l2 = 2 * l, N = L * L;
    const size_t total = (size_t)8 * 4 * 4 * 2 * l * l2;
    const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    const int i = (int)(gid % l2);
    size_t rest = gid / l2;
    const int dy = (int)(rest % l);
    rest /= l;
    const int sy = (int)(rest % 2);
    rest /= 2;
    const int comp = (int)(rest % 4);
    rest /= 4;
    const int kap = (int)(rest % 4);
    const int c = (int)(rest / 4);
    const int Kx = kap & 1, Ky = kap >> 1;
    const int x = i + c;
    double v = 0.0;
    if (x < l2) {
        const int xx = x % l;
        for (int F = 0; F < 4; ++F) {
            const int Fx = F & 1, Fy = F >> 1;
            const double w = W64[(size_t)comp * N + (size_t)(dy + l * Fy) * L + (xx + l * Fx)];
            v += ((Kx * Fx + Ky * Fy) & 1) ? -w : w;
        }
        if (x < l && Kx) v = -v;
        if (sy && Ky) v = -v;
    }
    const float f = (float)v;
    const __nv_bfloat16 hi = __float2bfloat16_rn(f);
    const __nv_bfloat16 lo = __float2bfloat16_rn(f - __bfloat162float(hi));
    const size_t base = ((((size_t)c * 4 + kap) * 4 + comp) * 2 + sy) * 2 * l * l2 + (size_t)dy * l2 + i;
    t2[base] = hi;
    t2[base + (size_t)l * l2] = lo;
}

// Spin spectra S'[r][kappa][a][e'] (bf16 hi/lo), e' = ey*l + (l-1-ex), of every cell offset.
__global__ void k_spec2_init(int L, int R, const float *__restrict__ spins, __nv_bfloat16 *hi,
                             __nv_bfloat16 *lo) {
    const int l = L / 2, lsq = l * l, N = L * L;
    const size_t total = (size_t)R * 12 * lsq;
    const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    const int ep = (int)(gid % lsq);
    const size_t ka = (gid / lsq) % 12, r = gid / ((size_t)12 * lsq);
    const int kap = (int)(ka / 3), a = (int)(ka % 3), Kx = kap & 1, Ky = kap >> 1;
    const int ey = ep / l, ex = l - 1 - (ep - ey * l);
    const float *s = spins + (r * 3 + a) * N;
    float v = 0.0f;
    for (int D = 0; D < 4; ++D) {
        const int Dx = D & 1, Dy = D >> 1;
        const float x = s[(ey + l * Dy) * L + ex + l * Dx];
        v += ((Kx * Dx + Ky * Dy) & 1) ? -x : x;
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[gid] = h;
    lo[gid] = __float2bfloat16_rn(v - __bfloat162float(h));
}
}  // namespace

size_t tc_wsh_elems(int L) { return (size_t)8 * 4 * 2 * L * 2 * L; }

size_t tc_t2_elems(int l) { return (size_t)8 * 4 * 4 * 2 * 2 * l * 2 * l; }

bool tc_spec2_supported(int L, int l, int Sw) { return L == 2 * l && l % 8 == 0 && (Sw == 256 || Sw == 512); }

cudaError_t launch_build_t2(int L, const double *W64, __nv_bfloat16 *t2, cudaStream_t st) {
    const int l = L / 2;
    const size_t total = (size_t)8 * 4 * 4 * 2 * l * 2 * l;
    k_build_t2<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(L, W64, t2);
    return cudaGetLastError();
}

cudaError_t launch_spec2_init(int L, int R, const float *spins, __nv_bfloat16 *hi, __nv_bfloat16 *lo, cudaStream_t st) {
    const size_t total = (size_t)R * 12 * (L / 2) * (L / 2);
    k_spec2_init<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(L, R, spins, hi, lo);
    return cudaGetLastError();
}

bool tc_supported(int L, int l, int B) {
    if (L % 8 || L < 8 || l < 2 || L % l) return false;
    const int n = (L / l) * (L / l);
    const int Sw = B * n;
    return Sw % 128 == 0 && (l * l) % B == 0;
}

size_t tc_smem_bytes() { return (size_t)kStages * kStage; }

cudaError_t launch_build_wsh(int L, const double *W64, __nv_bfloat16 *wsh, cudaStream_t st) {
    const size_t total = (size_t)8 * 4 * L * 2 * L;
    k_build_wsh<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(L, W64, wsh);
    return cudaGetLastError();
}

int tc_plan(int L, int Sw, int R, int nsm, TcUnit *units, int max_units, int *NT_out, int *tmem_cols,
            int *tile_first, int *mtiles_out, int *ntiles_out, bool spec2, int kblocks, int ntile) {
    const int N = L * L;
    const int cap = (ntile >= 16 && ntile <= 256) ? (ntile / 16) * 16 : 256;
    const int NT = R >= cap ? cap : ((R + 15) / 16) * 16;
    const int ntiles = (R + NT - 1) / NT;
    const int mt_inplane = 2 * Sw / 128, mt_zz = Sw / 128;
    // K per tile: Toeplitz rows contract (a, m) over 2N (in-plane) or N (zz); spectra
    // contract (a, e') or (kappa pair, e') over 2 l^2 = N / 2
    // (a spectra zz tile of a 512-site window holds one kappa, B = S_w/4 >= 128 rows: only its
    // half of the pair's K range, kappa % 2, is nonzero)
    const bool zz_one = spec2 && Sw / 4 >= 128;
    const int kb_inplane = spec2 ? N / 2 / kKB : 2 * N / kKB, kb_zz = spec2 ? (zz_one ? N / 4 : N / 2) / kKB : N / kKB;
    const long long total = (long long)ntiles * (mt_inplane * kb_inplane + mt_zz * kb_zz);
    // smallest K-blocks per unit whose units (rounded up per tile) fit one wave
    int kbpu = (int)((total + nsm - 1) / nsm);
    if (kbpu < (spec2 ? 4 : 2)) kbpu = spec2 ? 4 : 2;   // spectra: at least 4 K-blocks a unit (measured)
    if (kblocks > 0) kbpu = std::min(kblocks, kb_inplane);
    for (; kblocks <= 0; ++kbpu) {
        long long cnt = 0;
        for (int mt = 0; mt < mt_inplane + mt_zz; ++mt) {
            const int nkb = mt < mt_inplane ? kb_inplane : kb_zz;
            cnt += (nkb + kbpu - 1) / kbpu;
        }
        if (cnt * ntiles <= nsm || kbpu >= kb_inplane) break;
    }
    int nu = 0;
    const int mtiles = mt_inplane + mt_zz;
    for (int nt = 0; nt < ntiles; ++nt)
        for (int mt = 0; mt < mtiles; ++mt) {
            tile_first[nt * mtiles + mt] = nu;
            const int nkb = mt < mt_inplane ? kb_inplane : kb_zz;
            const int kb0 = (mt >= mt_inplane && zz_one) ? ((mt - mt_inplane) & 1) * kb_zz : 0;
            for (int kb = 0; kb < nkb; kb += kbpu) {
                if (nu >= max_units) return -1;
                units[nu].mtile = mt;
                units[nu].ntile = nt;
                units[nu].kb_begin = kb0 + kb;
                units[nu].kb_end = kb0 + (kb + kbpu < nkb ? kb + kbpu : nkb);
                ++nu;
            }
        }
    tile_first[ntiles * mtiles] = nu;
    *mtiles_out = mtiles;
    *ntiles_out = ntiles;
    *NT_out = NT;
    int cols = 32;
    while (cols < NT) cols <<= 1;
    *tmem_cols = cols;
    return nu;
}

// 2D tensor map of a [R][3N] bf16 spin (or spectra) array: boxes of kKB = 32 elements
// (64 bytes) x NT rows, written to shared memory in the 64-byte swizzled layout.  The
// driver's encoder is reached through the runtime's entry-point query, so the
// library does not link libcuda and loads on hosts without a driver.
int tc_encode_map(void *map, const __nv_bfloat16 *spins, int L, int R, int NT) {
    // looked up once per process (a function-local static: initialised once, even when
    // several host threads drive handles of their own)
    static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    if (!encode) return -1;
    const cuuint64_t dims[2] = {(cuuint64_t)3 * L * L, (cuuint64_t)R};
    const cuuint64_t strides[1] = {(cuuint64_t)3 * L * L * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {(cuuint32_t)kKB, (cuuint32_t)NT};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = encode(static_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                                              const_cast<__nv_bfloat16 *>(spins), dims, strides, box, estr,
                                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

size_t tc_map_bytes() { return sizeof(CUtensorMap); }

cudaError_t launch_tc_field(const TcFieldArgs &a, int nunits, const void *map_hi, const void *map_lo, cudaStream_t st) {
    const size_t smem = tc_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_tc_field, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(nunits);
    cfg.blockDim = dim3(kTcThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_tc_field, a, *static_cast<const CUtensorMap *>(map_hi),
                              *static_cast<const CUtensorMap *>(map_lo));
}

}  // namespace dipmc
