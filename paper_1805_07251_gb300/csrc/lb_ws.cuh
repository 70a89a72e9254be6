// lb_ws.cuh -- warp-specialised, persistent form of the fused D2Q9 step for one lane pair
// (two FP32 components, FP32-class mu), the same arithmetic as step_tile_pair in
// lb_kernels.cuh (bitwise the same results).
//
// A CTA of 12 warps walks a fixed list of 32 x 8 tiles (tile k of the CTA is
// blockIdx.x + k * gridDim.x).  Its warps have two roles:
//   loader warps (4)   phase 1 of tile k+1: the tile's own populations into shared memory,
//                      their densities, the densities of the 2-node ring;
//   compute warps (8)  phases 2 and 3 of tile k: mu on tile + 1 ring, then forces,
//                      friction, Psi, collision and push streaming to global memory.
// The stage of a tile (populations, densities) is double buffered; the hand-over uses
// named barriers (PTX bar.sync / bar.arrive):
//   FULL[b]   the loaders arrive when buffer b holds tile k, the compute warps wait on it;
//   EMPTY[b]  the compute warps arrive when they have read buffer b for the last time,
//             the loaders wait on it before filling it with tile k+2;
//   MU        the compute warps alone, between the mu phase and the collision.
// The mu array has one buffer: every compute thread arrives at FULL of tile k only after
// its collision of tile k-1, so no mu of tile k is written while tile k-1 still reads.
// Every barrier phase has exactly the 384 (FULL, EMPTY) or 256 (MU) threads of its
// count, and both roles run the same number of iterations (their CTA's tile count), so
// every wait ends.  The global loads of a tile thus overlap the arithmetic of the
// previous one instead of stalling the warps that do the arithmetic.
//
// Measured on GB300 (D2Q9, two components, 1024^2, double-float mu) it is slower than the
// tile kernel: 56.2 us per step against 46.8 us with 4 loader warps and three CTAs per SM
// (24 compute warps), 75.6 us with 2 loader warps and four CTAs per SM: the loads, issued
// by few warps, cannot keep up, and registers cap the warps an SM can hold.  It stays as
// an opt-in organisation (LB_KERNEL_WS).
#pragma once
#include "lb_kernels.cuh"

namespace lbvdw {

constexpr int WS_TX = 32, WS_TY = 8;
constexpr int WS_COMPUTE = WS_TX * WS_TY;  // 256 compute threads, one per tile node
constexpr int WS_LOADERS = 128;            // 4 loader warps
constexpr int WS_THREADS = WS_COMPUTE + WS_LOADERS;
constexpr int WS_BAR_FULL = 1, WS_BAR_EMPTY = 3, WS_BAR_MU = 5;  // named barrier ids (0: __syncthreads)

// named barriers with immediate ids, so that the kernel reserves only the ids it uses
template <int ID, int COUNT>
__device__ __forceinline__ void named_bar_sync() {
    asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(COUNT) : "memory");
}

template <int ID, int COUNT>
__device__ __forceinline__ void named_bar_arrive() {
    asm volatile("bar.arrive %0, %1;" ::"n"(ID), "n"(COUNT) : "memory");
}

// the FULL / EMPTY barrier of buffer b
__device__ __forceinline__ void ws_wait_full(int b) {
    if (b == 0) named_bar_sync<WS_BAR_FULL, WS_THREADS>();
    else named_bar_sync<WS_BAR_FULL + 1, WS_THREADS>();
}
__device__ __forceinline__ void ws_signal_full(int b) {
    if (b == 0) named_bar_arrive<WS_BAR_FULL, WS_THREADS>();
    else named_bar_arrive<WS_BAR_FULL + 1, WS_THREADS>();
}
__device__ __forceinline__ void ws_wait_empty(int b) {
    if (b == 0) named_bar_sync<WS_BAR_EMPTY, WS_THREADS>();
    else named_bar_sync<WS_BAR_EMPTY + 1, WS_THREADS>();
}
__device__ __forceinline__ void ws_signal_empty(int b) {
    if (b == 0) named_bar_arrive<WS_BAR_EMPTY, WS_THREADS>();
    else named_bar_arrive<WS_BAR_EMPTY + 1, WS_THREADS>();
}

// shared-memory layout (bytes) of one CTA
template <int MU>
struct WsLayout {
    using G = TileGeom<2, WS_TX, WS_TY>;
    using PT = typename std::conditional<MU == MU_DF, float4, float2>::type;
    static constexpr int Q = 9;
    static constexpr size_t g_bytes = (size_t)Q * WS_COMPUTE * sizeof(float2);    // own populations
    static constexpr size_t rho_bytes = (size_t)G::EY * G::EX * sizeof(float2);  // tile + 2 ring
    static constexpr size_t phi_bytes = (size_t)G::MY * G::MX * sizeof(PT);      // tile + 1 ring
    static constexpr size_t off_g = 0;
    static constexpr size_t off_rho = off_g + 2 * g_bytes;
    static constexpr size_t off_phi = off_rho + 2 * rho_bytes;
    static constexpr size_t off_tbl = off_phi + phi_bytes;
    static constexpr size_t bytes = off_tbl + TblWords<MU>::value * sizeof(float);
};

template <int FORCE, int MU>
__global__ void __launch_bounds__(WS_THREADS, 3)
    lb_step_ws_kernel(const float *__restrict__ fin, float *__restrict__ fout, DevParams P, int tiles_x, int ntiles) {
    using L = Lat<2>;
    using G = TileGeom<2, WS_TX, WS_TY>;
    using Lay = WsLayout<MU>;
    using PT = typename Lay::PT;
    constexpr int Q = L::Q, EX = G::EX, MX = G::MX, MY = G::MY, NT = WS_COMPUTE;
    static_assert(MU == MU_DF || MU == MU_F32, "lane pairs need an FP32-class mu");
    extern __shared__ __align__(16) unsigned char smem[];
    float *s_tbl = reinterpret_cast<float *>(smem + Lay::off_tbl);

    const int nx = P.nx, ny = P.ny;
    const int tid = threadIdx.x;
    load_tables<MU>(s_tbl, P, tid, WS_THREADS);
    __syncthreads();

    const size_t plane = (size_t)nx * (size_t)ny;
    const size_t cq = (size_t)Q * plane;  // component stride
    const bool small = nx <= WS_TX + 1 || ny <= WS_TY + 1;
    const float2 rref = make_float2(P.rho_ref_f[0], P.rho_ref_f[1]);
    const int count = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (tid >= NT) {
        // ------------------------------ loader warps: phase 1 of each tile -------------------
        const int lt = tid - NT;
        for (int it = 0; it < count; ++it) {
            const int b = it & 1;
            const int tile = (int)blockIdx.x + it * (int)gridDim.x;
            const int x0 = (tile % tiles_x) * WS_TX, y0 = (tile / tiles_x) * WS_TY;
            if (it >= 2) ws_wait_empty(b);  // compute warps are done with b
            float2 *s_g = reinterpret_cast<float2 *>(smem + Lay::off_g + b * Lay::g_bytes);
            float2 *s_rho = reinterpret_cast<float2 *>(smem + Lay::off_rho + b * Lay::rho_bytes);
            // own nodes n = lt + h * WS_LOADERS (whole tile rows per loader warp)
#pragma unroll
            for (int h = 0; h < NT / WS_LOADERS; ++h) {
                const int n = lt + h * WS_LOADERS;
                const int tx = n % WS_TX, ty = n / WS_TX;
                const int x = x0 + tx, y = y0 + ty;
                const int gx = small ? wrap(x, nx) : wrap1(x, nx);
                const int gy = small ? wrap(y, ny) : wrap1(y, ny);
                const float *src = fin + (size_t)gy * nx + gx;
                float2 gv[Q], acc, jx, jy;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    gv[i] = make_float2(src[(size_t)i * plane], src[cq + (size_t)i * plane]);
                    s_g[i * NT + n] = gv[i];
                }
                moments_lane<2>(gv, acc, jx, jy);
                s_rho[(ty + 2) * EX + tx + 2] = v_add(rref, acc);
            }
            // densities on the 2-node ring
            for (int k = lt; k < G::RING; k += WS_LOADERS) {
                int ex, ey;
                G::ring_node(k, ex, ey);
                const int gx = small ? wrap(x0 + ex - 2, nx) : wrap1(x0 + ex - 2, nx);
                const int gy = small ? wrap(y0 + ey - 2, ny) : wrap1(y0 + ey - 2, ny);
                const float *src = fin + (size_t)gy * nx + gx;
                float2 acc = make_float2(src[0], src[cq]);
#pragma unroll
                for (int i = 1; i < Q; ++i) acc = v_add(acc, make_float2(src[(size_t)i * plane], src[cq + (size_t)i * plane]));
                s_rho[ey * EX + ex] = v_add(rref, acc);
            }
            ws_signal_full(b);  // buffer b holds this tile
        }
        return;
    }

    // ------------------------------ compute warps: phases 2 and 3 ------------------------
    const int tx = tid % WS_TX, ty = tid / WS_TX;
    unsigned bad = 0;
    for (int it = 0; it < count; ++it) {
        const int b = it & 1;
        const int tile = (int)blockIdx.x + it * (int)gridDim.x;
        const int x0 = (tile % tiles_x) * WS_TX, y0 = (tile / tiles_x) * WS_TY;
        const float2 *s_g = reinterpret_cast<const float2 *>(smem + Lay::off_g + b * Lay::g_bytes);
        const float2 *s_rho = reinterpret_cast<const float2 *>(smem + Lay::off_rho + b * Lay::rho_bytes);
        PT *s_phi = reinterpret_cast<PT *>(smem + Lay::off_phi);
        ws_wait_full(b);  // the loaders have filled buffer b
        // the node's bare momenta, held through the mu phase (as the tile kernel does)
        float2 jx0, jy0;
        {
            float2 gv[Q], acc;
#pragma unroll
            for (int i = 0; i < Q; ++i) gv[i] = s_g[i * NT + tid];
            moments_lane<2>(gv, acc, jx0, jy0);
        }

        // ---- phase 2: phi on tile + 1 ring (as step_tile_pair) ---------------------------
        auto mu_at = [&](int k, bool store) {
            const int mx = k % MX, my = k / MX;
            const int e = (my + 1) * EX + mx + 1;
            float2 r[1], lp[1], lin[1];
            r[0] = s_rho[e];
            lp[0] = lap_d2q9(nbr9(s_rho + e, EX));
            lin_pairs<1>(r, lp, P, lin);
            bool ok;
            if constexpr (MU == MU_DF) {
                DF<float2> ph[1];
                ok = mu_pairs_df<1, FORCE>(r, lin, P, reinterpret_cast<const float4 *>(s_tbl), ph);
                if (store) s_phi[k] = make_float4(ph[0].hi.x, ph[0].hi.y, ph[0].lo.x, ph[0].lo.y);
            } else {
                float2 ph[1];
                ok = mu_pairs_f32<1, FORCE>(r, lin, P, ph);
                if (store) s_phi[k] = ph[0];
            }
            return ok || !store;
        };
        static_assert(MX * MY > NT && MX * MY <= 2 * NT, "two mu rounds");
        if ((tid & ~31) + NT < MX * MY) {
            const bool has2 = tid + NT < MX * MY;
            const bool ok1 = mu_at(tid, true);
            const bool ok2 = mu_at(has2 ? tid + NT : tid, has2);
            if (!(ok1 && ok2)) bad = 1;
        } else if (!mu_at(tid, true)) {
            bad = 1;
        }
        named_bar_sync<WS_BAR_MU, NT>();

        // ---- phase 3: forces, collision, streaming --------------------------------------
        const int x = x0 + tx, y = y0 + ty;
        if (x < nx && y < ny) {
            const int e = (ty + 2) * EX + tx + 2;
            const int m = (ty + 1) * MX + tx + 1;
            auto phi_at = [&](int k) {
                if constexpr (MU == MU_DF) {
                    const float4 t = s_phi[k];
                    return DF<float2>{make_float2(t.x, t.y), make_float2(t.z, t.w)};
                } else {
                    return s_phi[k];
                }
            };
            float2 rho[1], lap[1], grx[1], gry[1], gpx[1], gpy[1], jx[1], jy[1];
            rho[0] = s_rho[e];
            const Nbr9<float2> nb = nbr9(s_rho + e, EX);
            lap[0] = lap_d2q9(nb);
            if constexpr (!Flags<FORCE>::nid) grad_d2q9(nb, grx[0], gry[0]);
            else grx[0] = gry[0] = vc<float2>(0.0);
            grad_d2q9_diff(phi_diff2(phi_at(m + 1), phi_at(m - 1)), phi_diff2(phi_at(m + MX), phi_at(m - MX)),
                           phi_diff2(phi_at(m + MX + 1), phi_at(m - MX - 1)),  // NE - SW
                           phi_diff2(phi_at(m - MX + 1), phi_at(m + MX - 1)),  // SE - NW
                           vs(P.gkt3_f, rho[0]), vs(P.gkt12_f, rho[0]), gpx[0], gpy[0]);
            jx[0] = jx0, jy[0] = jy0;
            float2 gr[1][Q], post[1][Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) gr[0][i] = s_g[i * NT + tid];
            collide_pairs<2, 1, FORCE>(rho, lap, gpx, gpy, grx, gry, jx, jy, P, gr, post);
            const int xe = small ? wrap(x + 1, nx) : (x + 1 == nx ? 0 : x + 1);
            const int xw = small ? wrap(x - 1, nx) : (x == 0 ? nx - 1 : x - 1);
            const int yn = small ? wrap(y + 1, ny) : (y + 1 == ny ? 0 : y + 1);
            const int ys = small ? wrap(y - 1, ny) : (y == 0 ? ny - 1 : y - 1);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int cx = L::vx(i), cy = L::vy(i);
                const int dx = cx == 1 ? xe : (cx == -1 ? xw : x);
                const int dy = cy == 1 ? yn : (cy == -1 ? ys : y);
                float *dst = fout + (size_t)i * plane + (size_t)dy * nx + dx;
                dst[0] = post[0][i].x;
                dst[cq] = post[0][i].y;
            }
        }
        // the last reads of buffer b are done; the loaders may refill it
        // for iteration it + 2, if there is one
        if (it + 2 < count) ws_signal_empty(b);
    }
    if (bad) atomicOr(P.err, ERR_DOMAIN);
}

}  // namespace lbvdw
