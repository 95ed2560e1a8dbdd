// Paired 16-bit pipelined step (kernel 7): the 16-bit storage formats
// (deviations from a global or a per-cell reference density) with nx even.
//
// Same arithmetic, cell by cell and in the same order, as the other step
// variants (update_cell), so results are bit-identical to them; what changes
// is how the populations move:
//  * each thread owns two neighbouring cells along x, (x, x+1) with x even,
//    so one aligned 32-bit load brings a population of both cells: 19 loads
//    per two cells instead of per cell;
//  * a warp covers 64 cells of a row; a push along x shifts the pair by one
//    cell, so the destination word of a shifted population holds one value
//    of this thread and one of its neighbour lane, which arrives by a warp
//    shuffle: every lane then stores one aligned 32-bit word, and only the
//    first / last lane of the row add a 16-bit store for the value that
//    leaves the warp's span (the other half of that word belongs to the
//    neighbouring tile, which writes it in the same way);
//  * the psi ring rows are read as float2 pairs (19 shared loads per pair
//    for the 18 neighbours of both cells);
//  * the words of plane z+2 are loaded into registers while plane z is
//    collided; once they arrive the thread sums their densities into the
//    psi ring and parks the raw words in a two-plane shared-memory stash
//    (its own slots only, so no barrier), from which the collision of that
//    plane decodes them again two planes later.  Registers then hold one
//    plane of raw words instead of three.
// The one-cell ring of the tile comes through a three-stage cp.async buffer
// as aligned words: the top and bottom ring rows as whole words (two cells
// each), the left and right ring columns as the word holding the ring cell.
#pragma once
#include "step_kernel.cuh"

namespace lbm {

template <class Codec, int TY>
struct Pair16Layout {
    static constexpr int NT = 32 * TY;           // threads: one warp per tile row
    static constexpr int TXC = 64;               // cells per tile row
    static constexpr int PX = TXC + 4;           // psi row pitch: slot = x_local + 2 for x_local in [-1, 64]
    static constexpr int PLANE = PX * (TY + 2);
    static constexpr int NRW = TXC / 2 + 2;      // words of a ring row: x_local = -2 .. 65
    static constexpr int NH = 2 * NRW + 2 * TY;  // ring threads: row words, then left / right column cells
    static constexpr int NSTAGE = 3, NSLOT = 4;
    static constexpr bool kLocal = Codec::kLocal;
    static constexpr size_t stage_bytes = sizeof(uint32_t) * Q * NH;
    static constexpr size_t ref_stage_bytes = kLocal ? sizeof(float2) * NH : 0;
    static constexpr size_t psi_bytes = sizeof(float) * NSLOT * PLANE;
    static constexpr size_t rho_bytes = kLocal ? sizeof(float) * NSLOT * PLANE : 0;
    static constexpr size_t stash_bytes = sizeof(uint32_t) * 2 * Q * NT;          // raw words, two planes
    static constexpr size_t stash_ref_bytes = kLocal ? sizeof(float2) * 2 * NT : 0;  // their references
    static constexpr size_t bytes =
        NSTAGE * (stage_bytes + ref_stage_bytes) + psi_bytes + rho_bytes + stash_bytes + stash_ref_bytes;
    static_assert(NH <= NT, "tile too small for its ring");
    static_assert(PX % 2 == 0 && PLANE % 2 == 0 && stage_bytes % 8 == 0, "float2 alignment of the rings");
};

namespace pair16 {
template <class S>
__device__ __forceinline__ uint32_t bits(S v) {
    unsigned short b;
    memcpy(&b, &v, sizeof(b));
    return b;
}
template <class S>
__device__ __forceinline__ S from_bits(uint32_t w) {
    const unsigned short b = (unsigned short)(w & 0xffffu);
    S v;
    memcpy(&v, &b, sizeof(b));
    return v;
}
// the two 16-bit halves of a word (low: the pair's first cell)
template <class S>
__device__ __forceinline__ void halves(uint32_t w, S& lo, S& hi) {
    unsigned short l, h;
    asm("mov.b32 {%0, %1}, %2;" : "=h"(l), "=h"(h) : "r"(w));
    memcpy(&lo, &l, sizeof(l));
    memcpy(&hi, &h, sizeof(h));
}
}  // namespace pair16

template <class Codec, int COLL, int TY, class I>
__global__ void __launch_bounds__(32 * TY, (32 * TY >= 512) ? 1 : 512 / (32 * TY))
sc_step_pair16_kernel(const typename Codec::S* __restrict__ src, typename Codec::S* __restrict__ dst,
                      const StepArgs a) {
    using S = typename Codec::S;
    using R = float;
    using L = Pair16Layout<Codec, TY>;
    constexpr int PX = L::PX, PLANE = L::PLANE, NH = L::NH, NRW = L::NRW;
    constexpr bool LOCAL = L::kLocal;
    static_assert(sizeof(S) == 2, "16-bit storage only");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t* hstage = reinterpret_cast<uint32_t*>(smem_raw);                               // [NSTAGE][Q][NH]
    float2* rstage = reinterpret_cast<float2*>(smem_raw + L::NSTAGE * L::stage_bytes);      // [NSTAGE][NH]
    float* ring = reinterpret_cast<float*>(smem_raw + L::NSTAGE * (L::stage_bytes + L::ref_stage_bytes));
    float* rring = ring + L::NSLOT * PLANE;                                                 // rho (local)
    uint32_t* stash = reinterpret_cast<uint32_t*>(rring + (LOCAL ? L::NSLOT * PLANE : 0));  // [2][Q][NT]
    float2* stash_ref = reinterpret_cast<float2*>(stash + 2 * Q * L::NT);                  // [2][NT] (local)

    const int tid = threadIdx.x, lane = tid & 31, ly = tid >> 5;
    const R rho0 = a.rho0f, inv_rho0 = a.inv_rho0f;
    const DevParams dev = a.dev;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const I n = I(a.n), plane = I(nx) * I(ny);
    const int my_slot = (ly + 1) * PX + 2 * lane + 2;  // even: float2-aligned

    // Ring role of this thread (fixed): a word of the top / bottom ring row
    // (cells x_local = 2k-2, 2k-1), or the left / right ring column cell.
    int h_hy = 0, h_xl = 0, h_slot0 = -1, h_slot1 = -1;
    const bool h_on = tid < NH;
    if (h_on) {
        if (tid < 2 * NRW) {
            const int k = tid % NRW;
            h_hy = (tid < NRW) ? -1 : TY;
            h_xl = 2 * k - 2;  // x_local of the word's low cell
            const int row = (h_hy + 1) * PX;
            if (k >= 1) h_slot0 = row + h_xl + 2;
            if (k <= NRW - 2) h_slot1 = row + h_xl + 3;
        } else if (tid < 2 * NRW + TY) {  // left column: x_local = -1, high half of the word at -2
            h_hy = tid - 2 * NRW;
            h_xl = -2;
            h_slot1 = (h_hy + 1) * PX + 1;
        } else {  // right column: x_local = 64, low half of the word at 64
            h_hy = tid - 2 * NRW - TY;
            h_xl = 64;
            h_slot0 = (h_hy + 1) * PX + 66;
        }
    }

    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
        const int tile = item % a.n_tiles, chunk = item / a.n_tiles;
        const int x0 = (tile % a.tiles_x) * 64, y0 = (tile / a.tiles_x) * TY;
        const int zs = chunk * a.zchunk;
        const int ze = min(zs + a.zchunk, nz);

        const int gx = wrap_index(x0 + 2 * lane, nx), gy = wrap_index(y0 + ly, ny);  // gx even
        const bool row_on = y0 + ly < ny;                                            // warp-uniform
        const int last = min(31, (nx - x0) / 2 - 1);  // last lane whose pair lies in the box
        const bool pair_on = row_on && lane <= last;
        const I my_xy = I(gy) * I(nx) + I(gx);
        const I h_xy = h_on ? I(wrap_index(y0 + h_hy, ny)) * I(nx) + I(wrap_index(x0 + h_xl, nx)) : I(0);
        const int yp = (gy + 1 == ny) ? 0 : gy + 1, ym = (gy == 0) ? ny - 1 : gy - 1;
        const I yoff[3] = {I(ym) * I(nx), I(gy) * I(nx), I(yp) * I(nx)};
        // x of the 16-bit edge stores: the pair's right neighbour (cx = +1, last lane)
        // and left neighbour (cx = -1, lane 0), periodic
        const int x_right = (gx + 2 == nx) ? 0 : gx + 2;
        const int x_left = (gx == 0) ? nx - 1 : gx - 1;

        auto wrapz = [&](int z) { return z < 0 ? z + nz : (z >= nz ? z - nz : z); };
        auto stage_of = [&](int z) { return (z - zs + 1) % L::NSTAGE; };
        auto slot_of = [&](int z) { return (z - zs + 1) & (L::NSLOT - 1); };

        auto issue_halo = [&](int z) {
            if (h_on) {
                const I off = I(wrapz(z)) * plane + h_xy;
                uint32_t* st = hstage + stage_of(z) * (Q * NH);
                static_for<0, Q>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    async_copy::copy<4>(st + q * NH + tid, pop_at(src, q, n) + off);
                });
                if constexpr (LOCAL)
                    async_copy::copy<8>(rstage + stage_of(z) * NH + tid, a.ref_src + (I(wrapz(z)) * plane + h_xy));
            }
            async_copy::commit();
        };
        // density of one half of a raw word, summed in population order
        auto dens = [&](const uint32_t (&w)[Q], int hi, float ref) {
            R r = R(0);
            static_for<0, Q>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                S v0, v1;
                pair16::halves(w[q], v0, v1);
                const S v = hi ? v1 : v0;
                if constexpr (LOCAL) r += Codec::template decode_ref<q>(v, ref, dev);
                else r += Codec::template decode<q>(v, dev);
            });
            return r;
        };
        auto halo_psi = [&](int z) {
            if (h_on) {
                const uint32_t* st = hstage + stage_of(z) * (Q * NH);
                uint32_t w[Q];
                static_for<0, Q>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    w[q] = st[q * NH + tid];
                });
                float2 ref = make_float2(0.0f, 0.0f);
                if constexpr (LOCAL) ref = rstage[stage_of(z) * NH + tid];
                float* ps = ring + slot_of(z) * PLANE;
                float* rs = rring + slot_of(z) * PLANE;
                if (h_slot0 >= 0) {
                    const R r = dens(w, 0, ref.x);
                    ps[h_slot0] = psi_of<R>(r, rho0, inv_rho0);
                    if constexpr (LOCAL) rs[h_slot0] = r;
                }
                if (h_slot1 >= 0) {
                    const R r = dens(w, 1, ref.y);
                    ps[h_slot1] = psi_of<R>(r, rho0, inv_rho0);
                    if constexpr (LOCAL) rs[h_slot1] = r;
                }
            }
        };
        auto load_plane = [&](uint32_t (&w)[Q], float2& ref, int z) {
            const I off = I(wrapz(z)) * plane + my_xy;
            static_for<0, Q>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                w[q] = __ldg(reinterpret_cast<const uint32_t*>(pop_at(src, q, n) + off));
            });
            if constexpr (LOCAL) ref = __ldg(reinterpret_cast<const float2*>(a.ref_src + (I(wrapz(z)) * plane + my_xy)));
        };
        // psi (and density) of the pair's plane z into the rings, and its raw
        // words into the stash for the collision two planes later
        auto own_psi = [&](const uint32_t (&w)[Q], float2 ref, int z) {
            const R r0 = dens(w, 0, ref.x), r1 = dens(w, 1, ref.y);
            *reinterpret_cast<float2*>(ring + slot_of(z) * PLANE + my_slot) =
                make_float2(psi_of<R>(r0, rho0, inv_rho0), psi_of<R>(r1, rho0, inv_rho0));
            if constexpr (LOCAL) *reinterpret_cast<float2*>(rring + slot_of(z) * PLANE + my_slot) = make_float2(r0, r1);
            uint32_t* st = stash + (z & 1) * (Q * L::NT) + tid;
            static_for<0, Q>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                st[q * L::NT] = w[q];
            });
            if constexpr (LOCAL) stash_ref[(z & 1) * L::NT + tid] = ref;
        };

        // Force, collision and push of the pair of plane z (raw words in the stash).
        auto update_pair = [&](int z) {
            const uint32_t* w = stash + (z & 1) * (Q * L::NT) + tid;
            float2 ref = make_float2(0.0f, 0.0f);
            if constexpr (LOCAL) ref = stash_ref[(z & 1) * L::NT + tid];
            const float* pl[3] = {ring + slot_of(z - 1) * PLANE, ring + slot_of(z) * PLANE,
                                  ring + slot_of(z + 1) * PLANE};
            // psi around the pair: v[dz+1][dy+1][k] = psi at x_local = 2 lane - 2 + k
            float v[3][3][6];
            static_for<0, 9>([&](auto rc) {
                constexpr int dz = decltype(rc)::value / 3 - 1, dy = decltype(rc)::value % 3 - 1;
                const float2* rp = reinterpret_cast<const float2*>(pl[dz + 1] + my_slot + dy * PX - 2);
                const float2 m = rp[1];
                v[dz + 1][dy + 1][2] = m.x;
                v[dz + 1][dy + 1][3] = m.y;
                if constexpr (dy == 0 || dz == 0) {  // rows with neighbours at dx = -1, +1
                    const float2 l = rp[0], r = rp[2];
                    v[dz + 1][dy + 1][1] = l.y;
                    v[dz + 1][dy + 1][4] = r.x;
                    (void)l.x;
                    (void)r.y;
                }
            });
            R F[2][3];
            static_for<0, 2>([&](auto cc) {
                constexpr int c = decltype(cc)::value;
                // Eq. SC_force, in the order of update_cell
                R sx = R(0), sy = R(0), sz = R(0);
                static_for<1, Q>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    const R vq = v[cz(q) + 1][cy(q) + 1][2 + c + cx(q)];
                    if constexpr (cx(q) != 0) sx += R(wq(q) * cx(q)) * vq;
                    if constexpr (cy(q) != 0) sy += R(wq(q) * cy(q)) * vq;
                    if constexpr (cz(q) != 0) sz += R(wq(q) * cz(q)) * vq;
                });
                const R gpsi = -a.Gf * v[1][1][2 + c];
                F[c][0] = gpsi * sx;
                F[c][1] = gpsi * sy;
                F[c][2] = gpsi * sz;
            });

            const int zm = (z == 0) ? nz - 1 : z - 1;
            const int zn = (z + 1 == nz) ? 0 : z + 1;
            const I zoff[3] = {I(zm) * plane, I(z) * plane, I(zn) * plane};
            const float* rp3[3] = {rring + slot_of(z - 1) * PLANE, rring + slot_of(z) * PLANE,
                                   rring + slot_of(z + 1) * PLANE};
            uint32_t e[2][Q];  // encoded post-collision populations of the two cells
            static_for<0, 2>([&](auto cc) {
                constexpr int c = decltype(cc)::value;
                R f[Q];
                const float rf = c ? ref.y : ref.x;
                static_for<0, Q>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    S v0, v1;
                    pair16::halves(w[q * L::NT], v0, v1);
                    const S sv = c ? v1 : v0;
                    if constexpr (LOCAL) f[q] = Codec::template decode_ref<q>(sv, rf, dev);
                    else f[q] = Codec::template decode<q>(sv, dev);
                });
                if constexpr (COLL == COLL_SRT) collide_srt<R>(f, F[c][0], F[c][1], F[c][2], a.tauf, a.omegaf);
                else if constexpr (COLL == COLL_MRT) collide_mrt<R>(f, F[c][0], F[c][1], F[c][2], a.sf);
                else if constexpr (COLL == COLL_MRT_SPARSE)
                    collide_mrt_sparse<R, false>(f, F[c][0], F[c][1], F[c][2], a.sf);
                else if constexpr (COLL == COLL_MRT_SHEAR)
                    collide_mrt_sparse<R, false, false>(f, F[c][0], F[c][1], F[c][2], a.sf);
                else collide_mrt_sparse<R, true>(f, F[c][0], F[c][1], F[c][2], a.sf);
                static_for<0, Q>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    if constexpr (LOCAL) {
                        // deviation from the rest equilibrium at the destination's density
                        const float dref = rp3[cz(q) + 1][my_slot + c + cx(q) + cy(q) * PX];
                        e[c][q] = pair16::bits(Codec::template encode_ref<q>(f[q], dref, dev));
                    } else {
                        e[c][q] = pair16::bits(Codec::template encode<q>(f[q], dev));
                    }
                });
            });
            if constexpr (LOCAL) {  // this pair's density now: the reference of what it receives
                if (pair_on) {
                    const float2 rnow = *reinterpret_cast<const float2*>(rp3[1] + my_slot);
                    *reinterpret_cast<float2*>(a.ref_dst + (zoff[1] + my_xy)) = rnow;
                }
            }
            // Eq. LBE streaming: f_a(x + c_a, t + 1) = f*_a(x, t), as aligned words; each
            // store has its own lane condition, so the stores are predicated, not branched to
            static_for<0, Q>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                S* row = pop_at(dst, q, n) + (zoff[cz(q) + 1] + yoff[cy(q) + 1]);
                if constexpr (cx(q) == 0) {
                    if (pair_on) *reinterpret_cast<uint32_t*>(row + gx) = e[0][q] | (e[1][q] << 16);
                } else if constexpr (cx(q) > 0) {
                    // word (gx, gx+1) receives the left lane's second cell and this lane's first
                    const uint32_t from_left = __shfl_up_sync(0xffffffffu, e[1][q], 1);
                    if (pair_on && lane > 0) *reinterpret_cast<uint32_t*>(row + gx) = from_left | (e[0][q] << 16);
                    if (pair_on && lane == 0) row[gx + 1] = pair16::from_bits<S>(e[0][q]);
                    if (pair_on && lane == last) row[x_right] = pair16::from_bits<S>(e[1][q]);
                } else {
                    // word (gx, gx+1) receives this lane's second cell and the right lane's first
                    const uint32_t from_right = __shfl_down_sync(0xffffffffu, e[0][q], 1);
                    if (pair_on && lane < last) *reinterpret_cast<uint32_t*>(row + gx) = e[1][q] | (from_right << 16);
                    if (pair_on && lane == last) row[gx] = pair16::from_bits<S>(e[1][q]);
                    if (pair_on && lane == 0) row[x_left] = pair16::from_bits<S>(e[0][q]);
                }
            });
        };

        __syncthreads();  // the previous item's readers of the rings and the stash are done
        issue_halo(zs - 1);
        issue_halo(zs);
        issue_halo(zs + 1);
        uint32_t wf[Q];  // raw words of the plane in flight
        float2 rf = make_float2(0.0f, 0.0f);
        {
            uint32_t wb[Q];
            float2 rb = rf;
            load_plane(wf, rf, zs - 1);
            load_plane(wb, rb, zs);
            // psi of plane zs-1 (no collision: its stash slot is overwritten at once)
            own_psi(wf, rf, zs - 1);
            load_plane(wf, rf, zs + 1);
            own_psi(wb, rb, zs);
            own_psi(wf, rf, zs + 1);
        }
        async_copy::wait<2>();
        halo_psi(zs - 1);
        async_copy::wait<1>();
        halo_psi(zs);
        for (int z = zs; z < ze; ++z) {
            const bool more = z + 2 <= ze;
            if (more) {
                load_plane(wf, rf, z + 2);
                issue_halo(z + 2);
            } else {
                async_copy::commit();
            }
            async_copy::wait<1>();
            halo_psi(z + 1);
            __syncthreads();
            if (row_on) update_pair(z);
            // the thread's own stash slots of plane z are read: plane z+2 takes them
            if (more) own_psi(wf, rf, z + 2);
        }
    }
    async_copy::wait<0>();
}

}  // namespace lbm
