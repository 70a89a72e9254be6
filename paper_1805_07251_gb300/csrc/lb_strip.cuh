// lb_strip.cuh -- the fused D2Q9 step (Sec. III and V of Ridl & Wagner, the same
// arithmetic as lb_step_kernel in lb_kernels.cuh) organised as a streaming window.
//
// Each CTA owns a column strip TX nodes wide and a segment of its rows, and walks
// down the segment TY rows at a time.  The populations (FP32 deviations) of the
// rows ahead are fetched into shared memory by the bulk-copy (TMA) engine,
// cp.async.bulk with mbarrier completion, two row blocks ahead of the one being
// collided, so HBM traffic overlaps the arithmetic.  Densities and mu live in small
// shared-memory ring buffers: every row's rho and mu are computed once per CTA
// (the tile kernel recomputes a 2-node ring of rho and a 1-node ring of mu per
// tile), only the strip's side halos (2 columns of rho, 1 of mu) are computed twice.
//
// Row bookkeeping for a segment starting at row ys with K row blocks of TY rows:
//   population block b (b = 0..K) holds rows [ys + 2 + (b - 1) TY, ys + 2 + b TY)
//   and lives in slot b % 3; iteration k collides rows [ys + k TY, ys + (k+1) TY),
//   which needs population blocks k and k+1, rho on rows [y-2, y+TY+2) and mu on
//   rows [y-1, y+TY+1).  Block k+1's rows are exactly the rho rows that are new in
//   iteration k, and mu's new rows are [y+1, y+TY+1); the rest was computed in
//   iteration k-1 (or the prologue).  Block k+2 is in flight meanwhile.
#pragma once
#include "lb_kernels.cuh"

namespace lbvdw {

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy primitives (PTX ISA: mbarrier, cp.async.bulk)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// make the initialised barriers visible to the async proxy (the bulk-copy engine)
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic-proxy shared-memory accesses before later
// async-proxy (bulk-copy) accesses of the same memory
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte
// aligned), completing `bytes` transactions on the barrier
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes,
                                              unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bounded wait for the completion of the barrier's phase `parity`.  try_wait itself
// suspends the thread for a system-dependent time (~3.8 us per unsuccessful try on
// GB300, measured with lb_selftest_wait): the default 2^18 tries give up after about a
// second, far beyond any copy latency.  Returns false when the limit is reached.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity,
                                                  unsigned limit = 1u << 18) {
    for (unsigned it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ---------------------------------------------------------------------------
// stencils on three row pointers (rows y-1, y, y+1 of a ring buffer); the same
// arithmetic as grad_at / lap_at / grad_phi of lb_kernels.cuh (lb_lane.cuh)
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ Nbr9<T> nbr_rows(const T *s, const T *m, const T *n, int x) {
    return {m[x], m[x + 1], m[x - 1], n[x], s[x], n[x + 1], n[x - 1], s[x - 1], s[x + 1]};
}

template <class T>
__device__ __forceinline__ T lap_rows(const T *s, const T *m, const T *n, int x) {
    return lap_d2q9(nbr_rows(s, m, n, x));
}

template <class T>
__device__ __forceinline__ void grad_rows(const T *s, const T *m, const T *n, int x, T &gx, T &gy) {
    grad_d2q9(nbr_rows(s, m, n, x), gx, gy);
}

template <class R, class T>
__device__ __forceinline__ void grad_phi_rows(const T *s, const T *m, const T *n, int x, const DevParams &P, R &gx,
                                              R &gy) {
    R c3, c12, c2;
    phi_weights<R, T>(P, c3, c12, c2);
    grad_d2q9_diff(phi_diff<R>(m[x + 1], m[x - 1]), phi_diff<R>(n[x], s[x]),
                   phi_diff<R>(n[x + 1], s[x - 1]),  // NE - SW
                   phi_diff<R>(s[x + 1], n[x - 1]),  // SE - NW
                   c3, c12, gx, gy);
}

// ---------------------------------------------------------------------------
// shared-memory layout of one CTA
// ---------------------------------------------------------------------------
template <int N, int TX, int TY, int MU>
struct StripLayout {
    static constexpr int Q = 9, NQ = N * Q;
    static constexpr int PW = TX + 8;  // population row: columns x0-4 .. x0+TX+3 (16-byte aligned ends)
    static constexpr int RW = TX + 4;  // rho row: columns x0-2 .. x0+TX+1
    static constexpr int MW = TX + 2;  // mu row: columns x0-1 .. x0+TX
    static constexpr int RING = 16;    // rows held in the rho and mu rings
    static_assert(TY + 4 <= RING, "ring too short");
    static constexpr int NT = RW * TY;  // threads: one per new rho node of a row block
    using MT = typename MuStore<MU>::T;
    static constexpr size_t slot_floats = (size_t)NQ * TY * PW;
    static constexpr size_t slot_bytes = slot_floats * sizeof(float);
    static constexpr size_t off_pop = 0;
    static constexpr size_t off_rho = off_pop + 3 * slot_bytes;
    static constexpr size_t off_phi = off_rho + (size_t)N * RING * RW * sizeof(float);
    static constexpr size_t off_tbl = (off_phi + (size_t)N * RING * MW * sizeof(MT) + 15) / 16 * 16;
    static constexpr size_t off_bar = (off_tbl + TblWords<MU>::value * sizeof(float) + 7) / 8 * 8;
    static constexpr size_t bytes = off_bar + 4 * sizeof(unsigned long long);  // 3 barriers + abort word
};

// Issue the bulk copies of population block b of the segment starting at row ys into
// slot b % 3: for every plane and row, the columns x0-4 .. x0+TX+3 (periodically
// wrapped: up to three pieces).  Thread 0 posts the expected byte count.
template <int N, int TX, int TY, int MU>
__device__ __forceinline__ void strip_issue(const float *__restrict__ fin, float *pop, unsigned long long *bar,
                                            int b, int ys, int x0, int nx, int ny, size_t plane, int tid) {
    using Lay = StripLayout<N, TX, TY, MU>;
    constexpr int PW = Lay::PW;
    float *slot = pop + (size_t)(b % 3) * Lay::slot_floats;
    unsigned long long *sb = bar + (b % 3);
    if (tid == 0) mbar_arrive_expect_tx(sb, (unsigned)Lay::slot_bytes);
    const int row0 = ys + 2 + (b - 1) * TY;
    // the slot was last read through the generic proxy (before a CTA barrier); order
    // those reads before this thread's bulk writes into it
    if (tid < Lay::NQ * TY) fence_proxy_async();
    for (int job = tid; job < Lay::NQ * TY; job += Lay::NT) {
        const int p = job / TY, r = job - p * TY;
        int gy = row0 + r;
        gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
        const float *src_row = fin + (size_t)p * plane + (size_t)gy * nx;
        float *dst = slot + ((size_t)p * TY + r) * PW;
        int col = 0, gx = x0 - 4;
        gx = gx < 0 ? gx + nx : gx;
        while (col < PW) {
            int len = nx - gx;
            if (len > PW - col) len = PW - col;
            bulk_copy_g2s(dst + col, src_row + gx, (unsigned)len * 4u, sb);
            col += len;
            gx = 0;
        }
    }
}

// Densities rho^c on `rows` rows of population block b (from row r0 of the block)
// into the rho ring; thread t -> column t % RW, row t / RW.
template <int N, int TX, int TY, class R, int MU>
__device__ __forceinline__ void strip_rho(const float *pop, R *s_rho, const DevParams &P, int b, int r0, int rows,
                                          int tid) {
    using Lay = StripLayout<N, TX, TY, MU>;
    constexpr int RW = Lay::RW, PW = Lay::PW, RING = Lay::RING;
    if (tid >= RW * rows) return;
    const int cc = tid % RW, rr = r0 + tid / RW;
    const float *src = pop + (size_t)(b % 3) * Lay::slot_floats + (size_t)rr * PW + cc + 2;
    const int yy = 4 + (b - 1) * TY + rr;  // row - (ys - 2): the ring's row coordinate
    const int ring_row = yy & (RING - 1);
#pragma unroll
    for (int c = 0; c < N; ++c) {
        R acc = (R)src[(size_t)(c * Lay::Q) * TY * PW];
#pragma unroll
        for (int i = 1; i < Lay::Q; ++i) acc = v_add(acc, (R)src[(size_t)(c * Lay::Q + i) * TY * PW]);
        s_rho[((size_t)c * RING + ring_row) * RW + cc] = v_add(pv<R>(P.rho_ref[c], P.rho_ref_f[c]), acc);
    }
}

// phi^c (gamma mu^c, see mu_node) on `rows` rows starting at ring row coordinate yy0
// (row - (ys - 2)); thread t -> column t % MW, row t / MW.  Returns false on a domain error.
template <int N, int TX, int TY, class R, int FORCE, int MU>
__device__ __forceinline__ bool strip_mu(const R *s_rho, typename MuStore<MU>::T *s_phi, const float *s_tbl,
                                         const DevParams &P, int yy0, int rows, int tid) {
    using Lay = StripLayout<N, TX, TY, MU>;
    using MT = typename MuStore<MU>::T;
    constexpr int RW = Lay::RW, MW = Lay::MW, RING = Lay::RING;
    if (tid >= MW * rows) return true;
    const int cm = tid % MW, yy = yy0 + tid / MW;
    const int ex = cm + 1;  // rho ring column of this node
    const int rs = (yy - 1) & (RING - 1), rm = yy & (RING - 1), rn = (yy + 1) & (RING - 1);
    R r[N], lp[N], lin[N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
        const R *base = s_rho + (size_t)c * RING * RW;
        r[c] = base[rm * RW + ex];
        lp[c] = lap_rows<R>(base + rs * RW, base + rm * RW, base + rn * RW, ex);
    }
    lin_node<N, R>(r, lp, P, lin);
    MT phi[N];
    const bool ok = mu_node<N, R, FORCE, MU>(r, lin, P, s_tbl, phi);
#pragma unroll
    for (int c = 0; c < N; ++c) s_phi[((size_t)c * RING + rm) * MW + cm] = phi[c];
    return ok;
}

template <int N, int TX, int TY, class R, int FORCE, int MU>
__global__ void __launch_bounds__(StripLayout<N, TX, TY, MU>::NT, 2)
    lb_strip_kernel(const float *__restrict__ fin, float *__restrict__ fout, DevParams P, int segs) {
    using Lay = StripLayout<N, TX, TY, MU>;
    using MT = typename MuStore<MU>::T;
    using L = Lat<2>;
    constexpr int Q = 9, NT = Lay::NT, RW = Lay::RW, MW = Lay::MW, PW = Lay::PW, RING = Lay::RING;
    extern __shared__ __align__(128) unsigned char smem[];
    float *pop = reinterpret_cast<float *>(smem + Lay::off_pop);
    R *s_rho = reinterpret_cast<R *>(smem + Lay::off_rho);
    MT *s_phi = reinterpret_cast<MT *>(smem + Lay::off_phi);
    float *s_tbl = reinterpret_cast<float *>(smem + Lay::off_tbl);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem + Lay::off_bar);
    unsigned &s_abort = *reinterpret_cast<unsigned *>(bar + 3);

    const int nx = P.nx, ny = P.ny;
    const size_t plane = (size_t)nx * (size_t)ny;
    const int tid = threadIdx.x;
    const int strips = nx / TX;
    const int strip = blockIdx.x % strips, seg = blockIdx.x / strips;
    const int nblk = ny / TY;
    const int kb0 = (int)((long long)seg * nblk / segs), kb1 = (int)((long long)(seg + 1) * nblk / segs);
    const int K = kb1 - kb0;
    const int x0 = strip * TX, ys = kb0 * TY;

    if (tid == 0) {
        for (int s = 0; s < 3; ++s) mbar_init(bar + s, 1);
        fence_barrier_init();
        s_abort = 0;
    }
    load_tables<MU>(s_tbl, P, tid, NT);
    __syncthreads();
    if (K <= 0) return;

    strip_issue<N, TX, TY, MU>(fin, pop, bar, 0, ys, x0, nx, ny, plane, tid);
    strip_issue<N, TX, TY, MU>(fin, pop, bar, 1, ys, x0, nx, ny, plane, tid);
    int issued = 2;  // blocks 0 .. issued-1 are in flight or complete
    int waited = 0;  // blocks 0 .. waited-1 have completed
    unsigned bad = 0;

    // prologue: rho on rows [ys-2, ys+2) (the last 4 rows of block 0), mu on [ys-1, ys+1)
    // `waited` advances only past blocks whose wait succeeded, so that an abort drains
    // the block that timed out as well as every later one
    if (mbar_wait_bounded(bar + 0, 0)) waited = 1;
    else atomicOr(&s_abort, 1u);
    strip_rho<N, TX, TY, R, MU>(pop, s_rho, P, 0, TY - 4, 4, tid);
    __syncthreads();
    if (!strip_mu<N, TX, TY, R, FORCE, MU>(s_rho, s_phi, s_tbl, P, 1, 2, tid)) bad = 1;
    __syncthreads();

    for (int k = 0; k < K && !s_abort; ++k) {
        const int y = ys + k * TY;
        if (k + 2 <= K) {
            // slot (k+2) % 3 held block k-1, whose last reader passed the barrier
            // that ended iteration k-1
            strip_issue<N, TX, TY, MU>(fin, pop, bar, k + 2, ys, x0, nx, ny, plane, tid);
            issued = k + 3;
        }
        if (mbar_wait_bounded(bar + (k + 1) % 3, ((k + 1) / 3) & 1)) waited = k + 2;
        else atomicOr(&s_abort, 1u);
        // rho on the rows of block k+1: [y+2, y+TY+2)
        strip_rho<N, TX, TY, R, MU>(pop, s_rho, P, k + 1, 0, TY, tid);
        __syncthreads();
        // mu on rows [y+1, y+TY+1): ring coordinates (y+1) - (ys-2) = k TY + 3
        if (!strip_mu<N, TX, TY, R, FORCE, MU>(s_rho, s_phi, s_tbl, P, k * TY + 3, TY, tid)) bad = 1;
        __syncthreads();
        // collision of rows [y, y+TY) and push streaming
        if (tid < TX * TY) {
            const int col = tid % TX, row = tid / TX;
            const int x = x0 + col, gyr = y + row;
            const int yy = gyr - (ys - 2);
            const int rs = (yy - 1) & (RING - 1), rm = yy & (RING - 1), rn = (yy + 1) & (RING - 1);
            // population block and row of node row gyr: rows y, y+1 are the last two of block k
            const int bb = row < 2 ? k : k + 1;
            const int rr = row < 2 ? TY - 2 + row : row - 2;
            const float *src = pop + (size_t)(bb % 3) * Lay::slot_floats + (size_t)rr * PW + col + 4;
            R rho[N], lap[N], gpx[N], gpy[N], grx[N], gry[N], jx[N], jy[N], gr[N][Q], post[N][Q];
#pragma unroll
            for (int c = 0; c < N; ++c) {
                R acc;
#pragma unroll
                for (int i = 0; i < Q; ++i) gr[c][i] = (R)src[(size_t)(c * Q + i) * TY * PW];
                moments_lane<2>(gr[c], acc, jx[c], jy[c]);
                const R *rb = s_rho + (size_t)c * RING * RW;
                const int ex = col + 2;
                rho[c] = rb[rm * RW + ex];
                lap[c] = lap_rows<R>(rb + rs * RW, rb + rm * RW, rb + rn * RW, ex);
                if constexpr (!Flags<FORCE>::nid) grad_rows<R>(rb + rs * RW, rb + rm * RW, rb + rn * RW, ex, grx[c], gry[c]);
                else grx[c] = gry[c] = (R)0;
                const MT *pb = s_phi + (size_t)c * RING * MW;
                grad_phi_rows<R, MT>(pb + rs * MW, pb + rm * MW, pb + rn * MW, col + 1, P, gpx[c], gpy[c]);
            }
            collide_node<2, N, R, FORCE>(rho, lap, gpx, gpy, grx, gry, jx, jy, P, gr, post);
            const int xe = x + 1 == nx ? 0 : x + 1, xw = x == 0 ? nx - 1 : x - 1;
            const int gy = gyr;  // rows of a segment lie inside [0, ny)
            const int yn = gy + 1 == ny ? 0 : gy + 1, ysb = gy == 0 ? ny - 1 : gy - 1;
#pragma unroll
            for (int c = 0; c < N; ++c)
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int cx = L::vx(i), cy = L::vy(i);
                    const int dx = cx == 1 ? xe : (cx == -1 ? xw : x);
                    const int dy = cy == 1 ? yn : (cy == -1 ? ysb : gy);
                    fout[(size_t)(c * Q + i) * plane + (size_t)dy * nx + dx] = post[c][i];
                }
        }
        __syncthreads();
    }
    if (bad) atomicOr(P.err, ERR_DOMAIN);
    if (s_abort) {
        // let every copy that was issued land before the CTA's shared memory is released
        for (int b = waited; b < issued; ++b) mbar_wait_bounded(bar + b % 3, (b / 3) & 1);
        if (tid == 0) atomicOr(P.err, ERR_TIMEOUT);
    }
}

}  // namespace lbvdw
