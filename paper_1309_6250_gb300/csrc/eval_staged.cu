// eval_staged.cu -- the tricubic B-spline value / gradient / Laplacian evaluation of
// eval_bspline.cu (Appendix, Eq. b-splineapproximation; chain rule of Sec. II Coordinates;
// separate Laplacian table of Sec. III C) with the stencil rows staged in shared memory by
// the tensor memory accelerator (tiled cp.async.bulk.tensor copies, completion counted on
// mbarriers).  Used in pencil order (qmcspl_set_order), which is opt-in: on GB300 the
// cell-ordered gather kernel is faster for every workload measured.
//
// Order.  The positions are sorted into pencils of 2 x 2 grid cells in (x, y) and, within a
// pencil, by z cell (order.cu).  Every stencil of a pencil lies in one 5 x 5 block of (x, y)
// columns, so a z plane of that block -- 25 rows per table -- is the unit of staging, and
// sweeping a pencil in z needs each of its planes once.
//
// Pipeline.  A block (one per SM) takes work items (a pencil, or a z segment of one) in a
// static round-robin.  Its producer warp streams the planes an item needs, in z order, into
// a ring of S plane slots: one lane issues one tensor copy of the 5 x 5 box per table (split
// into in-range runs where the box wraps around the cell), and the slot's `full` barrier
// completes when all bytes have landed.  Each consumer warp takes every NC-th position of the
// item in order, waits for the four planes of that position, evaluates it from shared memory,
// and arrives on the `empty` barrier of every plane that no later position of its own needs;
// the producer refills a slot once all NC consumers have released it.  Consumers release a
// plane only after they have seen it full, so every copy has landed before its slot is reused
// and before the block exits.
//
// Rows per position read by the consumers: the same 64 per table as the gather kernel, but
// from shared memory; rows fetched from L2: 25 per plane, shared by the 2 x 2 cells of the
// pencil.  Results are bit-identical to the gather kernel (same weights, same products, same
// summation order).  What limits it: a plane of two FP32 tables of 128 orbitals is 25.6 KB, so
// the ring holds 8 planes, while the positions the consumer warps have in flight already span
// about 4 planes plus their z spread; the ring has little room left to prefetch, and fewer
// warps in flight hide less latency.
//
// Every wait is bounded (about a second of SM clock).  A wait that gives up sets bit 2 of the
// error word (QMCSPL_ERR_TIMEOUT at qmcspl_sync) and the abort flag that ends the other
// warps' waits; the producer still waits, again bounded, for its copies in flight before
// the block exits.
#include <cudaTypedefs.h>

#include <atomic>
#include <cstring>
#include <string>

#include "eval_common.cuh"
#include "staged.cuh"

namespace qmcspl {
namespace {

std::atomic<int> g_stall_launches{0};

constexpr long long kWaitCycles = 1LL << 31;   // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

#ifdef QMCSPL_DEBUG_BOUNDS
// count bytes that will not arrive (a copy skipped by the range check) as arrived
__device__ __forceinline__ void mbar_complete_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
#endif

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait, with all 32 lanes of the warp, for the completion of the phase with the given
// parity: at most kWaitCycles, and no longer once another warp has set the abort flag.  The
// lanes decide together (every lane polls; the warp goes on when all have seen the phase
// complete), so the result is the same in every lane and the warp never splits.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, volatile int* abort_flag, int* err)
{
    bool done = mbar_try_wait(bar, parity);
    if (__all_sync(kFullMask, done)) return true;
    const long long t0 = clock64();
    for (;;) {
        done = done || mbar_try_wait(bar, parity);
        if (__all_sync(kFullMask, done)) return true;
        int stop = *abort_flag ? 1 : (clock64() - t0 > kWaitCycles ? 2 : 0);
        stop = __shfl_sync(kFullMask, stop, 0);
        if (stop) {
            if (stop == 2 && (threadIdx.x & 31) == 0) {
                *abort_flag = 1;
                atomicOr(err, 4);
            }
            return false;
        }
    }
}

__device__ __forceinline__ uint4 lds16(uint32_t addr)
{
    uint4 r;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "r"(addr));
    return r;
}

__device__ __forceinline__ int wrapn(int x, int n)
{
    x %= n;
    return x < 0 ? x + n : x;
}

// One work item: positions [q0, q1) of the evaluation order, pencil (px, py), stored planes
// zlo .. zlo + n_planes - 1.
struct Item {
    long long q0, q1;
    int px, py, zlo, n_planes;
};

__device__ __forceinline__ int record_iz(const EvalArgs& p, long long q)
{
    const long long ip = order_index(p, q);
    const int c = __float_as_int(__ldg(static_cast<const float4*>(p.rec) + ip).x);
    return c >= 0 ? (c >> 20) & 1023 : 0;
}

__device__ __forceinline__ bool item_range(const EvalArgs& p, const StagedArgs& s, long long it, Item& r)
{
    const long long pencil = it / s.nseg;
    const int seg = (int)(it - pencil * s.nseg);
    const int z0 = seg * s.zseg;
    const int z1 = min(z0 + s.zseg, p.nz);
    const long long b0 = pencil * p.nz + z0, b1 = pencil * p.nz + z1;
    r.q0 = b0 > 0 ? __ldg(s.bin_end + b0 - 1) : 0;
    r.q1 = __ldg(s.bin_end + b1 - 1);
    r.px = (int)(pencil / s.npy);
    r.py = (int)(pencil - (long long)r.px * s.npy);
    r.zlo = 0;
    r.n_planes = 0;
    if (r.q1 <= r.q0) return false;
    // stored plane of stencil row z = iz - 1 is iz (one ghost plane below z = 0)
    r.zlo = record_iz(p, r.q0);
    r.n_planes = record_iz(p, r.q1 - 1) + 4 - r.zlo;
    return r.n_planes >= 4;
}

// One tiled tensor copy (TMA) of a box of the 4-D table view [x][y][z][orbital] into shared
// memory, completion counted on `bar`.  Coordinates innermost first: orbital (always 0), z, y, x.
__device__ __forceinline__ void tma_box(uint32_t dst, const CUtensorMap* map, int z, int y, int x, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(z), "r"(y), "r"(x), "r"(smem_addr(bar))
        : "memory");
}

// The periodic index range [s0, s0 + kBox) of an axis of N >= 4 points as at most two
// in-range runs: run j starts at index st[j], has len[j] points and lands at box offset at[j].
__device__ __forceinline__ int box_runs(int s0, int N, int* st, int* len, int* at)
{
    if (s0 < 0) {
        st[0] = N + s0; len[0] = -s0; at[0] = 0;
        st[1] = 0; len[1] = kBox + s0; at[1] = -s0;
        return 2;
    }
    if (s0 + kBox > N) {
        st[0] = s0; len[0] = N - s0; at[0] = 0;
        st[1] = 0; len[1] = s0 + kBox - N; at[1] = N - s0;
        return 2;
    }
    st[0] = s0; len[0] = kBox; at[0] = 0;
    return 1;
}

// Stage stored plane z of the pencil whose box starts at (x0, y0) for table t into the slot
// at shared address dst: the 5 x 5 rows, [x][y] row-major, one row per (x, y) column.  A box
// that does not wrap in y goes as one copy per x run (box kBox rows in y); one that wraps in
// y as one copy per x row and y run.  Called by one lane.
__device__ __forceinline__ void stage_plane(const StagedMaps& maps, const EvalArgs& p, const StagedArgs& s, int t,
                                            int z, int x0, int y0, uint32_t dst, uint64_t* bar)
{
    int xs[2], xl[2], xa[2], ys[2], yl[2], ya[2];
    const int nxr = box_runs(x0, p.nx, xs, xl, xa);
    const int nyr = box_runs(y0, p.ny, ys, yl, ya);
    const uint32_t rb = (uint32_t)s.row_bytes;
    if (nyr == 1) {
        for (int i = 0; i < nxr; ++i)
            tma_box(dst + (uint32_t)(xa[i] * kBox) * rb, &maps.m[t][xl[i] - 1], z, ys[0], xs[i], bar);
    } else {
        for (int xi = 0; xi < kBox; ++xi) {
            const int x = wrapn(x0 + xi, p.nx);
            for (int j = 0; j < nyr; ++j) {
                const int mi = yl[j] == kBox ? 0 : kBox + yl[j] - 1;   // box of 1 x row, yl[j] y rows
                tma_box(dst + (uint32_t)(xi * kBox + ya[j]) * rb, &maps.m[t][mi], z, ys[j], x, bar);
            }
        }
    }
}

__device__ void staged_producer(const EvalArgs& p, const StagedArgs& s, const StagedMaps& maps, uint64_t* full,
                                uint64_t* empty, unsigned char* ring, volatile int* abort_flag, int lane)
{
    const uint32_t slot_bytes = (uint32_t)s.n_tab * kPlaneRows * s.row_bytes;
    const uint32_t tab_bytes = (uint32_t)kPlaneRows * s.row_bytes;
    const uint32_t ring_addr = smem_addr(ring);
    long long issued = 0;
    bool ok = s.stall == 0;
    for (long long it = blockIdx.x; ok && it < s.n_items; it += gridDim.x) {
        Item r;
        if (!item_range(p, s, it, r)) continue;
        const int x0 = kPencilEdge * r.px - 1, y0 = kPencilEdge * r.py - 1;
        for (int k = 0; k < r.n_planes; ++k) {
            const long long q = issued;
            const int slot = (int)(q % s.slots);
            const long long fill = q / s.slots;
            if (fill > 0 && !mbar_wait(empty + slot, (unsigned)((fill - 1) & 1), abort_flag, p.err)) {
                ok = false;
                break;
            }
            if (lane == 0) {
                mbar_arrive_expect_tx(full + slot, slot_bytes);
                const int z = r.zlo + k;
#ifdef QMCSPL_DEBUG_BOUNDS
                if (z < 0 || z >= p.nz + 3) {   // stored planes are 0 .. nz + 2
                    atomicOr(p.err, 2);
                    mbar_complete_tx(full + slot, slot_bytes);
                } else
#endif
                    for (int t = 0; t < s.n_tab; ++t)
                        stage_plane(maps, p, s, t, z, x0, y0, ring_addr + (uint32_t)slot * slot_bytes + t * tab_bytes,
                                    full + slot);
            }
            __syncwarp();
            ++issued;
        }
    }
    // no copy may still be in flight when the block exits: wait for the last fill of each slot
    for (int slot = lane; slot < s.slots; slot += 32) {
        if (slot >= issued) break;
        const long long last = slot + ((issued - 1 - slot) / s.slots) * s.slots;
        const unsigned parity = (unsigned)((last / s.slots) & 1);
        if (!mbar_try_wait(full + slot, parity)) {
            const long long t0 = clock64();
            while (!mbar_try_wait(full + slot, parity)) {
                if (clock64() - t0 > kWaitCycles) {
                    atomicOr(p.err, 4);
                    break;
                }
            }
        }
    }
}

// Evaluate the position of this lane group from the staged planes.  sb[n]: shared address of
// the slot holding stored plane iz + n; xr, yr: the position's cell within the pencil (0, 1).
template <typename T, bool LAPTAB>
__device__ __forceinline__ void staged_position(const EvalArgs& p, const StagedArgs& s, long long ip, int sub,
                                                const uint32_t* sb, int xr, int yr, float tx, float ty,
                                                float tz)
{
    constexpr int E = Traits<T>::E;
    constexpr int NP = Pairs<T>::N;
    constexpr int R = LAPTAB ? 8 : 4;
    const uint32_t tabb = kPlaneRows * s.row_bytes;

    float bx[4], dbx[4], d2bx[4], by[4], dby[4], d2by[4], bz[4], dbz[4], d2bz[4];
    bspline_weights<float>(tx, bx, dbx, LAPTAB ? nullptr : d2bx);
    bspline_weights<float>(ty, by, dby, LAPTAB ? nullptr : d2by);
    bspline_weights<float>(tz, bz, dbz, LAPTAB ? nullptr : d2bz);
    f32x2 bz2[4], dbz2[4], d2bz2[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        bz2[n] = pack2(bz[n], bz[n]);
        dbz2[n] = pack2(dbz[n], dbz[n]);
        if (!LAPTAB) d2bz2[n] = pack2(d2bz[n], d2bz[n]);
    }
    float ml0 = 0.f, ml1 = 0.f, ml2 = 0.f, ml3 = 0.f, ml4 = 0.f, ml5 = 0.f;
    if (!LAPTAB) {
        ml0 = p.mlf[0]; ml1 = p.mlf[1]; ml2 = p.mlf[2];
        ml3 = p.mlf[3]; ml4 = p.mlf[4]; ml5 = p.mlf[5];
    }
    // row (l, m) of a plane: box column (xr + l, yr + m); this lane's 16-byte chunk
    const uint32_t lane_off = (uint32_t)sub * 16u;
    auto row_off = [&](int c) -> uint32_t {
        const int l = c >> 2, m = c & 3;
        return (uint32_t)((xr + l) * kBox + (yr + m)) * s.row_bytes + lane_off;
    };

    f32x2 V[NP], GX[NP], GY[NP], GZ[NP], LP[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) V[j] = GX[j] = GY[j] = GZ[j] = LP[j] = 0ull;

    uint4 cur[R], nxt[R];
    {
        const uint32_t o = row_off(0);
#pragma unroll
        for (int n = 0; n < 4; ++n) cur[n] = lds16(sb[n] + o);
        if (LAPTAB) {
#pragma unroll
            for (int n = 0; n < 4; ++n) cur[4 + n] = lds16(sb[n] + tabb + o);
        }
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        const int l = c >> 2, m = c & 3;
        if (c < 15) {   // next column's rows in flight while this one is contracted
            const uint32_t o = row_off(c + 1);
#pragma unroll
            for (int n = 0; n < 4; ++n) nxt[n] = lds16(sb[n] + o);
            if (LAPTAB) {
#pragma unroll
                for (int n = 0; n < 4; ++n) nxt[4 + n] = lds16(sb[n] + tabb + o);
            }
        }
        f32x2 A0[NP], A1[NP], A2[NP], AL[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) A0[j] = A1[j] = A2[j] = AL[j] = 0ull;
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            f32x2 cv[NP];
            Pairs<T>::get(cur[n], cv);
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                A0[j] = ffma2(bz2[n], cv[j], A0[j]);
                A1[j] = ffma2(dbz2[n], cv[j], A1[j]);
                if (!LAPTAB) A2[j] = ffma2(d2bz2[n], cv[j], A2[j]);
            }
            if (LAPTAB) {
                Pairs<T>::get(cur[4 + n], cv);
#pragma unroll
                for (int j = 0; j < NP; ++j) AL[j] = ffma2(bz2[n], cv[j], AL[j]);
            }
        }
        const float w00 = bx[l] * by[m], w10 = dbx[l] * by[m], w01 = bx[l] * dby[m];
        const f32x2 W00 = pack2(w00, w00), W10 = pack2(w10, w10), W01 = pack2(w01, w01);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            V[j] = ffma2(W00, A0[j], V[j]);
            GX[j] = ffma2(W10, A0[j], GX[j]);
            GY[j] = ffma2(W01, A0[j], GY[j]);
            GZ[j] = ffma2(W00, A1[j], GZ[j]);
        }
        if (LAPTAB) {
#pragma unroll
            for (int j = 0; j < NP; ++j) LP[j] = ffma2(W00, AL[j], LP[j]);
        } else {
            const float c0 = ml0 * (d2bx[l] * by[m]) + ml1 * (bx[l] * d2by[m]) + ml3 * (dbx[l] * dby[m]);
            const float c1 = ml4 * w10 + ml5 * w01;
            const float c2 = ml2 * w00;
            const f32x2 C0 = pack2(c0, c0), C1 = pack2(c1, c1), C2 = pack2(c2, c2);
#pragma unroll
            for (int j = 0; j < NP; ++j) LP[j] = ffma2(C0, A0[j], ffma2(C1, A1[j], ffma2(C2, A2[j], LP[j])));
        }
        if (c < 15) {
#pragma unroll
            for (int k = 0; k < R; ++k) cur[k] = nxt[k];
        }
    }

    const int o0 = sub * E;
    if (o0 >= p.n_orb) return;
    const bool vec = p.vec_out != 0;
    float v[E], gx[E], gy[E], gz[E], lp[E];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        unpack2(V[j], v[2 * j], v[2 * j + 1]);
        unpack2(GX[j], gx[2 * j], gx[2 * j + 1]);
        unpack2(GY[j], gy[2 * j], gy[2 * j + 1]);
        unpack2(GZ[j], gz[2 * j], gz[2 * j + 1]);
        unpack2(LP[j], lp[2 * j], lp[2 * j + 1]);
    }
    float cg[3][E];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float m0 = p.mgf[3 * a], m1 = p.mgf[3 * a + 1], m2 = p.mgf[3 * a + 2];
#pragma unroll
        for (int e = 0; e < E; ++e) cg[a][e] = fmaf(m0, gx[e], fmaf(m1, gy[e], m2 * gz[e]));
    }
    if (p.phase) bloch_apply<float, E>(p, ip, v, cg, lp, true, !LAPTAB);
    if (p.val) store_run<float, E>(static_cast<float*>(p.val) + ip * p.n_orb + o0, v, o0, p.n_orb, vec);
    if (p.grad) {
        float* g = static_cast<float*>(p.grad) + ip * 3 * p.n_orb + o0;
#pragma unroll
        for (int a = 0; a < 3; ++a) store_run<float, E>(g + (size_t)a * p.n_orb, cg[a], o0, p.n_orb, vec);
    }
    if (p.lap) store_run<float, E>(static_cast<float*>(p.lap) + ip * p.n_orb + o0, lp, o0, p.n_orb, vec);
}

__device__ __forceinline__ int warp_min(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(kFullMask, v, o));
    return v;
}
__device__ __forceinline__ int warp_max(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFullMask, v, o));
    return v;
}

// Consumer warp `cw` of `nc`.  With L lanes per position a warp task is G = 32 / L
// consecutive positions of the item (one per lane group).  If the task's planes do not fit
// in the ring at once, its groups are evaluated one round each.
template <typename T, bool LAPTAB>
__device__ void staged_consumer(const EvalArgs& p, const StagedArgs& s, uint64_t* full, uint64_t* empty,
                                const unsigned char* ring, volatile int* abort_flag, int cw, int nc, int lane)
{
    const int L = 1 << p.lanes_log2;
    const int G = 32 >> p.lanes_log2;
    const int sub = lane & (L - 1);
    const int grp = lane >> p.lanes_log2;
    const unsigned slot_bytes = (unsigned)s.n_tab * kPlaneRows * s.row_bytes;
    const uint32_t ring_addr = smem_addr(ring);
    long long seq = 0;   // planes of earlier items, in the producer's numbering
    // wait until plane (seq + r) is full, then (lane 0, after the warp) release it
    auto release = [&](int r) -> bool {
        const long long q = seq + r;
        const int slot = (int)(q % s.slots);
        if (!mbar_wait(full + slot, (unsigned)((q / s.slots) & 1), abort_flag, p.err)) return false;
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + slot);
        return true;
    };
    for (long long it = blockIdx.x; it < s.n_items; it += gridDim.x) {
        Item r;
        if (!item_range(p, s, it, r)) continue;
        const long long n = r.q1 - r.q0;
        int rel = 0;   // planes [0, rel) of this item are released by this warp
        // the next task's position and record are loaded one task ahead
        long long nip = 0;
        float4 nrec = make_float4(0.f, 0.f, 0.f, 0.f);
        auto fetch = [&](long long t) {
            const long long qi = t + grp;
            if (qi < n) {
                nip = order_index(p, r.q0 + qi);
                nrec = __ldg(static_cast<const float4*>(p.rec) + nip);
            }
        };
        fetch((long long)cw * G);
        for (long long t0 = (long long)cw * G; t0 < n; t0 += (long long)nc * G) {
            const bool act = t0 + grp < n;
            const long long ip = nip;
            const float4 rec = nrec;
            fetch(t0 + (long long)nc * G);
            int ix = 0, iy = 0, iz = 0;
            float tx = 0.f, ty = 0.f, tz = 0.f;
            bool ok = false;
            if (act) {
                unpack_cell(__float_as_int(rec.x), ix, iy, iz, ok);
                tx = rec.y;
                ty = rec.z;
                tz = rec.w;
            }
            const int r0 = iz - r.zlo, xr = ix - 2 * r.px, yr = iy - 2 * r.py;
            const bool in = act && r0 >= 0 && r0 + 4 <= r.n_planes && xr >= 0 && xr <= 1 && yr >= 0 && yr <= 1;
            if (act && sub == 0) {
                if (!ok) atomicOr(p.err, 1);
                if (!in) atomicOr(p.err, 2);   // not in this item's pencil: not evaluated
            }
            const int lo = warp_min(in ? r0 : 0x7fffffff);
            const int hi = warp_max(in ? r0 + 3 : -1);
            if (hi < 0) continue;
            const bool one_round = hi - lo + 1 <= s.slots;
            const int rounds = one_round ? 1 : G;
            for (int g = 0; g < rounds; ++g) {
                const bool mine = in && (one_round || g == grp);
                int rlo = one_round ? lo : warp_min(mine ? r0 : 0x7fffffff);
                if (rlo == 0x7fffffff) continue;
                const int rhi = one_round ? hi : rlo + 3;
                for (; rel < rlo; ++rel)
                    if (!release(rel)) return;
                for (int k = rlo; k <= rhi; ++k) {
                    const long long q = seq + k;
                    if (!mbar_wait(full + (int)(q % s.slots), (unsigned)((q / s.slots) & 1), abort_flag, p.err))
                        return;
                }
                if (mine) {
                    uint32_t sb[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) sb[k] = ring_addr + (uint32_t)((seq + r0 + k) % s.slots) * slot_bytes;
                    staged_position<T, LAPTAB>(p, s, ip, sub, sb, xr, yr, tx, ty, tz);
                }
                __syncwarp();
            }
        }
        for (; rel < r.n_planes; ++rel)
            if (!release(rel)) return;
        seq += r.n_planes;
    }
}

template <typename T, bool LAPTAB>
__global__ void __launch_bounds__(32 * (kStagedConsumers + 1), 1)
    bspline_vgl_staged_kernel(const EvalArgs p, const StagedArgs s, const __grid_constant__ StagedMaps maps)
{
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + s.slots;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + s.slots);
    unsigned char* ring = smem + kStagedRingOffset;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nc = (int)(blockDim.x >> 5) - 1;
    if (threadIdx.x == 0) {
        for (int i = 0; i < s.slots; ++i) {
            mbar_init(full + i, 1);
            mbar_init(empty + i, (unsigned)nc);
        }
        *abort_flag = 0;
        // make the initialised barriers visible to the asynchronous (bulk copy) proxy
        asm volatile("fence.mbarrier_init.release.cluster;\n\tfence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0) staged_producer(p, s, maps, full, empty, ring, abort_flag, lane);
    else staged_consumer<T, LAPTAB>(p, s, full, empty, ring, abort_flag, warp - 1, nc, lane);
}

template <typename T, bool LAPTAB>
int launch_staged_typed(const EvalArgs& a, const StagedArgs& s, const StagedMaps& maps, int consumers,
                        cudaStream_t st)
{
    auto kern = bspline_vgl_staged_kernel<T, LAPTAB>;
    const size_t smem = staged_smem_bytes(s);
    static thread_local int configured = -1;   // dynamic shared memory limit set per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured != dev) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kStagedMaxSmem);
        if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(staged kernel)");
        configured = dev;
    }
    long long blocks = sm_count();
    if (blocks > s.n_items) blocks = s.n_items;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, 32 * (consumers + 1), smem, st>>>(a, s, maps);
    return cuda_error(cudaGetLastError(), "bspline_vgl_staged_kernel launch");
}

// cuTensorMapEncodeTiled from the driver, through the runtime (no link to the driver library);
// null when the driver does not provide it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// The tensor maps of the handle's staged tables: the table as the 4-D array
// [x][y][z][orbital] (z over the stored planes, ghost planes included), one map per box shape.
int encode_maps(const Handle* h, const StagedArgs& s, StagedMaps* maps)
{
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return set_error(QMCSPL_ERR_CUDA, "the driver does not provide cuTensorMapEncodeTiled");
    const cuuint64_t rb = (cuuint64_t)s.row_bytes;
    const cuuint64_t dims[4] = {(cuuint64_t)h->n_orb_p, (cuuint64_t)h->rows_z, (cuuint64_t)h->dims[1],
                                (cuuint64_t)h->dims[0]};
    const cuuint64_t strides[3] = {rb, rb * h->rows_z, rb * h->rows_z * (cuuint64_t)h->dims[1]};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt =
        h->storage == QMCSPL_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    std::memset(maps, 0, sizeof(*maps));
    for (int t = 0; t < s.n_tab; ++t) {
        void* base = const_cast<void*>(h->table(t));
        for (int i = 0; i < kStagedMaps; ++i) {
            const cuuint32_t by = i < kBox ? kBox : (cuuint32_t)(i - kBox + 1);
            const cuuint32_t bx = i < kBox ? (cuuint32_t)(i + 1) : 1;
            const cuuint32_t box[4] = {(cuuint32_t)h->n_orb_p, 1, by, bx};
            const CUresult r = enc(&maps->m[t][i], dt, 4, base, dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS)
                return set_error(QMCSPL_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
        }
    }
    return QMCSPL_OK;
}

}  // namespace

bool staged_eligible(const Handle* h)
{
    if (h->method != QMCSPL_BSPLINE_SMOOTH && h->method != QMCSPL_BSPLINE_INTERP) return false;
    if (is_general(h) || h->separate_grad || h->tiles != 1) return false;
    if (h->storage != QMCSPL_F32 && h->storage != QMCSPL_BF16) return false;
    const long long rb = (long long)h->n_orb_p * (long long)h->elem_bytes;
    if (rb != 16LL << h->lanes_log2 || rb % 128 != 0 || rb > 512) return false;
    if (!tensor_map_encoder()) return false;
    const long long n_tab = h->separate_lap ? 2 : 1;
    const long long slots = (kStagedMaxSmem - kStagedRingOffset) / (n_tab * kPlaneRows * rb);
    return slots >= kStagedMinSlots;
}

bool staged_plan(const Handle* h, long long n_pos, BinGeometry* g, StagedArgs* s)
{
    const int npx = (h->dims[0] + kPencilEdge - 1) / kPencilEdge;
    const int npy = (h->dims[1] + kPencilEdge - 1) / kPencilEdge;
    const long long n_pencils = (long long)npx * npy;
    const long long n_bins = n_pencils * h->dims[2];
    if (n_bins > kMaxPencilBins || n_pos >= (1LL << 31) - 1) return false;
    g->edge[0] = g->edge[1] = kPencilEdge;
    g->edge[2] = 1;
    g->nb[0] = npx;
    g->nb[1] = npy;
    g->nb[2] = h->dims[2];
    g->n_bins = (int)n_bins;
    // about 30 work items per block balance the static schedule; a z segment shorter
    // than 16 cells would re-stage too many of its 3 overhang planes
    long long nseg = (30LL * sm_count() + n_pencils / 2) / n_pencils;
    const long long max_seg = h->dims[2] / 16 > 1 ? h->dims[2] / 16 : 1;
    if (nseg > max_seg) nseg = max_seg;
    if (nseg < 1) nseg = 1;
    s->zseg = (int)((h->dims[2] + nseg - 1) / nseg);
    s->nseg = (h->dims[2] + s->zseg - 1) / s->zseg;
    s->npx = npx;
    s->npy = npy;
    s->n_items = n_pencils * s->nseg;
    s->elem_bytes = (int)h->elem_bytes;
    s->row_bytes = h->n_orb_p * (int)h->elem_bytes;
    s->n_tab = h->separate_lap ? 2 : 1;
    long long slots = (kStagedMaxSmem - kStagedRingOffset) / ((long long)s->n_tab * kPlaneRows * s->row_bytes);
    if (slots > kStagedMaxSlots) slots = kStagedMaxSlots;
    s->slots = (int)slots;
    s->bin_end = nullptr;
    return slots >= kStagedMinSlots;
}

bool use_staged(const Handle* h, long long n_pos)
{
    // opt-in only: on GB300 the cell-ordered gather kernel is faster for every workload
    // measured (its L1 keeps more of the shared stencil rows than the shared-memory ring)
    (void)n_pos;
    return h->order_mode == QMCSPL_ORDER_PENCIL && staged_eligible(h);
}

int launch_bspline_vgl_staged(const Handle* h, const Prepared& pr, long long n_pos, void* val, void* grad,
                              void* lap, StagedArgs s, cudaStream_t st)
{
    EvalArgs a;
    fill_eval_args(h, &a);
    a.rec = pr.rec;
    a.perm = pr.perm;
    a.phase = pr.phase;
    a.n_pos = n_pos;
    a.val = val;
    a.grad = grad;
    a.lap = lap;
    const uintptr_t al = (uintptr_t)val | (uintptr_t)grad | (uintptr_t)lap;
    a.vec_out = ((h->n_orb * 4) % 16 == 0) && (al % 16 == 0);   // FP32 outputs
    s.bin_end = pr.bin_end;
    s.stall = 0;
    for (int v = g_stall_launches.load(); v > 0;)
        if (g_stall_launches.compare_exchange_weak(v, v - 1)) {
            s.stall = 1;
            break;
        }
    if (!a.rec || !a.perm || !s.bin_end) return set_error(QMCSPL_ERR_ARG, "staged evaluation needs the pencil order");
    static thread_local StagedMaps maps;   // 2.3 KB: off the stack
    const int rc = encode_maps(h, s, &maps);
    if (rc != QMCSPL_OK) return rc;
    const int nc = kStagedConsumers;
    const bool lt = h->separate_lap != 0;
    if (h->storage == QMCSPL_F32)
        return lt ? launch_staged_typed<float, true>(a, s, maps, nc, st)
                  : launch_staged_typed<float, false>(a, s, maps, nc, st);
    return lt ? launch_staged_typed<__nv_bfloat16, true>(a, s, maps, nc, st)
              : launch_staged_typed<__nv_bfloat16, false>(a, s, maps, nc, st);
}

}  // namespace qmcspl

extern "C" int qmcspl_debug_stall_pipeline(int n)
{
    qmcspl::g_stall_launches.store(n > 0 ? n : 0);
    return QMCSPL_OK;
}
