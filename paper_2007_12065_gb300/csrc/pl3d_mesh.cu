// pl3d_mesh.cu -- the explicit half-edge mesh of a frame (Algorithm 1: T and T_map; Algorithm 2:
// HE) and the triangle lists and boundary half-edges of its planar segments (the inputs of the
// polygon extraction of Section 7.2), in one cooperative launch (pl3d_extract_mesh).
//
// Phases, one grid barrier apart, all over chunks of 1024 consecutive entries (4 per thread:
// consecutive ones in the sort, one per round of 256 consecutive GIDs in A and C):
//   A  per chunk of GIDs: valid triangles (all three points valid, Algorithm 1) and segment
//      roots (a label is the smallest GID of its segment, so a root is labelled with itself),
//      kept as ballot words (no scan phase: each CTA sums the counts of the chunks before its own
//      when it needs them)
//   C  T, T_map and the segment index of each root, in GID order
//   D  HE from the neighbours' T_map (the twin rules of Algorithm 2) and the boundary half-edges
//      (no twin, or a twin of another label); sort keys: the segment index of each T entry (the
//      segment count for an unlabelled one, so it sorts last)
//   With at most kMaxOnePass segments, the lists come from one counting pass instead of a sort:
//   D also counts the entries of each (segment, chunk of T) pair into a segments x chunks matrix
//   (zeroed in C; warp-aggregated atomics), then
//   S  each segment's row becomes its exclusive prefix over the chunks, and the row total its size
//   P  a stable scatter straight into the segment lists: an entry's place is its segment's start,
//      plus its row's prefix at its chunk, plus the entries of its segment in the chunk's earlier
//      warps and its rank among equal segments in its warp (__match_any_sync); the CSR offsets
//      are the segment starts
//   With more segments:
//   R  a stable LSD radix sort of (segment index, T index) with digits of up to 8 bits: per-chunk
//      digit histograms; per-digit exclusive scans over the chunks; a stable scatter that ranks
//      equal digits inside a warp with __match_any_sync and across warps with per-warp counters
//   G  the segments' CSR (offsets where the key changes)
// Data written by one CTA and read by another after a barrier is loaded with __ldcg (L2), never
// through the non-coherent read-only path.
// Everything in T order keeps GID order, so the lists come out sorted by (label, T index).
#include <string.h>

#include <algorithm>

#include "pl3d_ctx.cuh"
#include "sync.cuh"

namespace pl3d {
namespace mesh {

constexpr int kChunk = 1024;
constexpr int kPer = kChunk / kThreads;   // 4 consecutive entries per thread
constexpr int kMaxDigitBits = 8;   // radix digits of up to 8 bits (11-bit digits, one pass below 2048 segments, measured slower)
constexpr int kMaxBins = 1 << kMaxDigitBits;
constexpr int kWarps = kThreads / 32;
// one counting pass up to this many segments: their starts and per-warp counts in shared memory
constexpr int kMaxOnePass = 2048;
constexpr size_t kSmemRadix = 2 * kMaxBins * sizeof(int) + (size_t)kWarps * kMaxBins * sizeof(uint16_t);
constexpr size_t kSmemOnePass = kMaxOnePass * sizeof(int) + (size_t)kWarps * kMaxOnePass * sizeof(uint16_t);
constexpr size_t kSmemBytes = kSmemRadix > kSmemOnePass ? kSmemRadix : kSmemOnePass;
static_assert(kMaxOnePass % kThreads == 0, "segment starts: the same count per thread");

struct MeshArgs {
    const float* points;
    const int32_t* labels;       // nullptr: no segment outputs
    int H, W;
    int32_t* T;                  // [3 |T|]
    int32_t* Tmap;               // [2Q]
    int32_t* HE;                 // [3 |T|]
    long long* counts;           // [3]: |T|, segments, triangles in segments
    int32_t* seg_labels;         // [segments]
    int32_t* seg_offsets;        // [segments + 1]
    int32_t* seg_tris;           // [triangles in segments]
    uint8_t* border;             // [|T|]
    int n_chunks;                // chunks of GIDs
    int32_t* cnt;                // [2][n_chunks]: T entries and roots per chunk -> exclusive offsets
    unsigned* bits;              // [2][n_chunks kChunk / 32]: valid triangles, segment roots, one bit per GID
    int32_t* root_idx;           // [2Q]
    int32_t* keys[2];            // [2Q]
    int32_t* vals[2];            // [2Q]
    int32_t* hist;               // [kMaxBins][n_chunks]
    int32_t* bin_tot;            // [kMaxBins]
    int32_t* seg_chunk;          // [segments][chunks of T, padded to 8]: entries per (segment, chunk) -> row prefixes
    int32_t* seg_cnt;            // [kMaxOnePass]: entries per segment
    long long seg_chunk_cap;     // entries of seg_chunk
    unsigned* barrier;
    int* error;
};

__device__ __forceinline__ bool vertex_valid(const float* P, long long i) {
    return point_valid(__ldg(P + 3 * i), __ldg(P + 3 * i + 1), __ldg(P + 3 * i + 2));
}

// Vertex (point) indices of triangle gid in the order of Algorithm 1:
// first = {p3, p2, p1}, second = {p1, p4, p3}.
__device__ __forceinline__ void tri_vertices(long long gid, int W, int Wq, long long v[3]) {
    const int q = (int)(gid >> 1);   // 2 (H - 1)(W - 1) < 2^31
    const int u = q / Wq, c = q - u * Wq;
    const long long p1 = (long long)u * W + c, p2 = p1 + 1, p3 = p1 + W + 1, p4 = p1 + W;
    if ((gid & 1) == 0) {
        v[0] = p3, v[1] = p2, v[2] = p1;
    } else {
        v[0] = p1, v[1] = p4, v[2] = p3;
    }
}

// Exclusive prefix of v over the CTA (thread order); *total receives the sum. Uses sh[kWarps + 1].
__device__ __forceinline__ int block_exclusive(int v, int* sh, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < kWarps; ++w) {
            const int t = sh[w];
            sh[w] = run;
            run += t;
        }
        sh[kWarps] = run;
    }
    __syncthreads();
    const int r = sh[warp] + x - v;
    *total = sh[kWarps];
    __syncthreads();
    return r;
}

// Sums of a and b over the CTA, in every thread (one barrier to publish, one before sh is reused).
// Uses sh[2 kWarps].
__device__ __forceinline__ void block_sum2(int a, int b, int* sh, int* ta, int* tb) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wa = (int)__reduce_add_sync(0xffffffffu, (unsigned)a), wb = (int)__reduce_add_sync(0xffffffffu, (unsigned)b);
    if (lane == 0) {
        sh[warp] = wa;
        sh[kWarps + warp] = wb;
    }
    __syncthreads();
    int sa = 0, sb = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        sa += sh[w];
        sb += sh[kWarps + w];
    }
    *ta = sa;
    *tb = sb;
    __syncthreads();
}

struct Flags {
    bool valid, root;
};

__device__ __forceinline__ Flags gid_flags(const MeshArgs& a, long long g, long long n) {
    Flags f = {false, false};
    if (g >= n) return f;
    long long v[3];
    tri_vertices(g, a.W, a.W - 1, v);
    // the three points and the label loaded together (no short circuit between them)
    const bool v0 = vertex_valid(a.points, v[0]), v1 = vertex_valid(a.points, v[1]), v2 = vertex_valid(a.points, v[2]);
    const int lab = a.labels ? __ldg(a.labels + g) : -1;
    f.valid = v0 & v1 & v2;
    f.root = f.valid && lab == (int)g;
    return f;
}

__global__ void __launch_bounds__(kThreads, 4) mesh_kernel(const __grid_constant__ MeshArgs a) {
    __shared__ int sh_scan[kWarps + 1];
    __shared__ int sh_sum[2 * kWarps];
    // dynamic: digit counts [kMaxBins], digit bases [kMaxBins], per-warp digit counts
    // [kWarps][kMaxBins] (16-bit: at most kChunk / kWarps entries per warp)
    extern __shared__ int mesh_smem[];
    int* const sh_bins = mesh_smem;
    int* const sh_base = mesh_smem + kMaxBins;
    uint16_t* const sh_wc = reinterpret_cast<uint16_t*>(mesh_smem + 2 * kMaxBins);
    const int Wq = a.W - 1, Hq = a.H - 1;
    const long long n = 2LL * Hq * Wq;
    const int C = a.n_chunks;
    int32_t* cT = a.cnt;
    int32_t* cR = a.cnt + C;

    // A: counts per chunk; every GID's root index starts undefined. A chunk is kPer rounds of
    // kThreads consecutive GIDs (thread t takes GID t of each round), so a warp's loads and
    // stores cover consecutive triangles.
    for (int c = blockIdx.x; c < C; c += gridDim.x) {
        const long long c0 = (long long)c * kChunk;
        int nt = 0, nr = 0;
        Flags fl[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) fl[j] = gid_flags(a, c0 + j * kThreads + threadIdx.x, n);   // loads in flight together
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const long long g = c0 + j * kThreads + threadIdx.x;
            const Flags f = fl[j];
            nt += f.valid;
            nr += f.root;
            if (a.labels && g < n) a.root_idx[g] = -1;
            // the flags as bits, one word per warp and round (kept for phase C)
            const unsigned bv = __ballot_sync(0xffffffffu, f.valid), br = __ballot_sync(0xffffffffu, f.root);
            if ((threadIdx.x & 31) == 0) {
                const long long w = (c0 + j * kThreads + threadIdx.x) >> 5;
                a.bits[w] = bv;
                a.bits[(long long)C * (kChunk / 32) + w] = br;
            }
        }
        int tt, tr;
        block_sum2(nt, nr, sh_sum, &tt, &tr);
        if (threadIdx.x == 0) {
            cT[c] = tt;
            cR[c] = tr;
        }
    }
    grid_barrier(a.barrier, a.error);

    // every CTA sums the chunk counts it needs itself (no separate scan phase): the totals, and
    // below the counts of the chunks before each of its own
    long long nT, nS_l;
    {
        long long st = 0, sr = 0;
        for (int i = threadIdx.x; i < C; i += blockDim.x) {
            st += __ldcg(cT + i);
            sr += __ldcg(cR + i);
        }
        int tt, tr;
        block_sum2((int)st, (int)sr, sh_sum, &tt, &tr);
        nT = tt;
        nS_l = tr;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.counts[0] = nT;
            a.counts[1] = nS_l;
            a.counts[2] = 0;
        }
    }
    const int nS = (int)nS_l;
    const int Ct = (int)((nT + kChunk - 1) / kChunk);   // chunks of T entries
    const int Ctp = (Ct + 7) & ~7;   // the matrix's row stride: rows start on 32-byte boundaries
    // the lists from one counting pass (S, P) instead of the radix sort (R, G)
    const bool one = a.labels && a.seg_chunk && nS > 0 && nS <= kMaxOnePass && (long long)nS * Ctp <= a.seg_chunk_cap;

    // C: T, T_map, segment roots (GID order). A GID's place among the chunk's entries
    // is the count of (round, warp) blocks before its own plus its lane's rank in its warp's
    // ballot; the per-block counts live in sh_wc (free until the sort).
    constexpr int kBlocks = kPer * kWarps;   // (round, warp) blocks of a chunk
    static_assert(kBlocks <= 64 && 4 * kBlocks <= kWarps * kMaxBins / 2, "block counts: two per lane of warp 0");
    int* const cntT = reinterpret_cast<int*>(sh_wc);
    int* const cntR = cntT + kBlocks;
    int* const preT = cntT + 2 * kBlocks;
    int* const preR = cntT + 3 * kBlocks;
    for (int c = blockIdx.x; c < C; c += gridDim.x) {
        const long long c0 = (long long)c * kChunk;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        Flags f[kPer];
        unsigned bv[kPer], brt[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const long long w = (c0 + j * kThreads) / 32 + warp;
            bv[j] = __ldcg(a.bits + w);
            brt[j] = __ldcg(a.bits + (long long)C * (kChunk / 32) + w);
            f[j].valid = (bv[j] >> lane) & 1u;
            f[j].root = (brt[j] >> lane) & 1u;
        }
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                cntT[j * kWarps + warp] = __popc(bv[j]);
                cntR[j * kWarps + warp] = __popc(brt[j]);
            }
        }
        long long bt = 0, br = 0;   // entries of the chunks before c
        for (int i = threadIdx.x; i < c; i += blockDim.x) {
            bt += __ldcg(cT + i);
            br += __ldcg(cR + i);
        }
        int ct, cr;
        block_sum2((int)bt, (int)br, sh_sum, &ct, &cr);   // (its barriers also publish the counts above)
        if (warp == 0) {   // exclusive prefix over the (round, warp) blocks, two per lane
            const int k0 = 2 * lane;
            const int t0 = k0 < kBlocks ? cntT[k0] : 0, t1 = k0 + 1 < kBlocks ? cntT[k0 + 1] : 0;
            const int r0 = k0 < kBlocks ? cntR[k0] : 0, r1 = k0 + 1 < kBlocks ? cntR[k0 + 1] : 0;
            int st = t0 + t1, sr = r0 + r1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int yt = __shfl_up_sync(0xffffffffu, st, o), yr = __shfl_up_sync(0xffffffffu, sr, o);
                if (lane >= o) {
                    st += yt;
                    sr += yr;
                }
            }
            if (k0 < kBlocks) {
                preT[k0] = st - (t0 + t1);
                preR[k0] = sr - (r0 + r1);
            }
            if (k0 + 1 < kBlocks) {
                preT[k0 + 1] = st - t1;
                preR[k0 + 1] = sr - r1;
            }
        }
        __syncthreads();
        const unsigned below = (1u << lane) - 1u;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const long long g = c0 + j * kThreads + threadIdx.x;
            if (g >= n) continue;
            const int k = j * kWarps + warp;
            if (f[j].valid) {
                const int pt = ct + preT[k] + __popc(bv[j] & below);
                long long v[3];
                tri_vertices(g, a.W, Wq, v);
                a.T[3LL * pt] = (int32_t)v[0];
                a.T[3LL * pt + 1] = (int32_t)v[1];
                a.T[3LL * pt + 2] = (int32_t)v[2];
                a.Tmap[g] = pt;
            } else {
                a.Tmap[g] = -1;
            }
            if (f[j].root) {
                const int pr = cr + preR[k] + __popc(brt[j] & below);
                a.seg_labels[pr] = (int32_t)g;
                a.root_idx[g] = pr;
            }
        }
        __syncthreads();   // the next chunk rewrites the block counts
    }
    if (one) {   // the (segment, chunk) counts start at zero, the rows' padding included
        const long long nz = (long long)nS * Ctp;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nz; i += (long long)gridDim.x * blockDim.x)
            a.seg_chunk[i] = 0;
    }
    grid_barrier(a.barrier, a.error);

    // D: HE (Algorithm 2) and the sort keys
    {
        const long long stride = (long long)gridDim.x * blockDim.x;
        for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (long long)Hq * Wq; q += stride) {
            const int u = (int)(q / Wq), v = (int)(q - (long long)u * Wq);
            const int32_t* tm = a.Tmap;
            // every load of the quad issued up front (none waits on another's value): its two
            // T_map entries and its neighbours' across its four outer edges, and the labels of
            // the same triangles (GIDs 2q, 2q + 1 and the neighbours')
            const bool hasr = v + 1 < Wq, hast = u > 0, hasl = v > 0, hasb = u + 1 < Hq;
            const int first = __ldcg(tm + 2 * q), second = __ldcg(tm + 2 * q + 1);
            const int right = hasr ? __ldcg(tm + 2 * (q + 1) + 1) : -1;
            const int top = hast ? __ldcg(tm + 2 * (q - Wq) + 1) : -1;
            const int left = hasl ? __ldcg(tm + 2 * (q - 1)) : -1;
            const int bottom = hasb ? __ldcg(tm + 2 * (q + Wq)) : -1;
            const int32_t* const L = a.labels;
            const int l1 = L ? __ldg(L + 2 * q) : -1, l2 = L ? __ldg(L + 2 * q + 1) : -1;
            const bool bd = a.border && L;
            const int lr = bd && hasr ? __ldg(L + 2 * (q + 1) + 1) : -1;
            const int lt = bd && hast ? __ldg(L + 2 * (q - Wq) + 1) : -1;
            const int ll = bd && hasl ? __ldg(L + 2 * (q - 1)) : -1;
            const int lb = bd && hasb ? __ldg(L + 2 * (q + Wq)) : -1;
            if (first >= 0) {
                a.HE[3LL * first] = right >= 0 ? 3 * right : -1;
                a.HE[3LL * first + 1] = top >= 0 ? 3 * top + 1 : -1;
                a.HE[3LL * first + 2] = second >= 0 ? 3 * second + 2 : -1;
            }
            if (second >= 0) {
                a.HE[3LL * second] = left >= 0 ? 3 * left : -1;
                a.HE[3LL * second + 1] = bottom >= 0 ? 3 * bottom + 1 : -1;
                a.HE[3LL * second + 2] = first >= 0 ? 3 * first + 2 : -1;
            }
            if (a.border) {
                // a half-edge is on a segment's boundary when it has no twin or the twin's label
                // differs; unlabelled triangles have no boundary
                if (first >= 0) {
                    unsigned bits = 0;
                    if (l1 >= 0) {
                        bits |= (right < 0 || lr != l1) ? 1u : 0u;
                        bits |= (top < 0 || lt != l1) ? 2u : 0u;
                        bits |= (second < 0 || l2 != l1) ? 4u : 0u;
                    }
                    a.border[first] = (uint8_t)bits;
                }
                if (second >= 0) {
                    unsigned bits = 0;
                    if (l2 >= 0) {
                        bits |= (left < 0 || ll != l2) ? 1u : 0u;
                        bits |= (bottom < 0 || lb != l2) ? 2u : 0u;
                        bits |= (first < 0 || l1 != l2) ? 4u : 0u;
                    }
                    a.border[second] = (uint8_t)bits;
                }
            }
            if (a.labels && nS > 0) {
                for (int side = 0; side < 2; ++side) {
                    const int t = side == 0 ? first : second;
                    int key = nS;
                    if (t >= 0) {
                        // the segment index of the label's root; a label that names no root (only
                        // possible for labels not made by pl3d_extract_planes) sorts with the rest
                        const int l = side == 0 ? l1 : l2;
                        const int k = (l >= 0 && l < n) ? __ldcg(a.root_idx + l) : -1;
                        key = k >= 0 ? k : nS;
                        a.keys[0][t] = key;
                        if (!one) a.vals[0][t] = t;
                    }
                    if (one) {
                        // entries per (segment, chunk of T): one atomic per group of equal cells
                        // among the warp's active lanes
                        const int cell = (t >= 0 && key < nS) ? key * Ctp + t / kChunk : -1;
                        const unsigned peers = __match_any_sync(__activemask(), cell);
                        if (cell >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1)
                            atomicAdd(a.seg_chunk + cell, __popc(peers));
                    }
                }
            }
        }
    }
    if (!a.labels || nS == 0) {
        // no segments: no lists (the boundary flags are all 0)
        if (a.labels && blockIdx.x == 0 && threadIdx.x == 0) a.seg_offsets[0] = 0;
        return;
    }
    grid_barrier(a.barrier, a.error);

    if (one) {
        const int ln = threadIdx.x & 31, wp = threadIdx.x >> 5;
        // S: each segment's row of chunk counts becomes its exclusive prefix, and the row total
        // the segment's size: a warp per row, in spans of 256 chunks, 8 consecutive per lane (two
        // 16-byte loads; the padding past Ct is zero), scanned in registers and then across the
        // lanes, carried from span to span
        {
            for (int k = blockIdx.x * kWarps + wp; k < nS; k += gridDim.x * kWarps) {
                int32_t* const row = a.seg_chunk + (long long)k * Ctp;
                int carry = 0;
                for (int base = 0; base < Ctp; base += 32 * 8) {
                    const int c0 = base + 8 * ln;
                    int4 u = make_int4(0, 0, 0, 0), w = u;
                    if (c0 < Ctp) {
                        u = __ldcg(reinterpret_cast<const int4*>(row + c0));
                        w = __ldcg(reinterpret_cast<const int4*>(row + c0 + 4));
                    }
                    const int e1 = u.x, e2 = e1 + u.y, e3 = e2 + u.z, e4 = e3 + u.w;   // exclusive in the lane
                    const int e5 = e4 + w.x, e6 = e5 + w.y, e7 = e6 + w.z, local = e7 + w.w;
                    int x = local;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, x, o);
                        if (ln >= o) x += y;
                    }
                    const int r0 = carry + x - local;
                    if (c0 < Ctp) {
                        *reinterpret_cast<int4*>(row + c0) = make_int4(r0, r0 + e1, r0 + e2, r0 + e3);
                        *reinterpret_cast<int4*>(row + c0 + 4) = make_int4(r0 + e4, r0 + e5, r0 + e6, r0 + e7);
                    }
                    carry += __shfl_sync(0xffffffffu, x, 31);
                }
                if (ln == 0) a.seg_cnt[k] = carry;
            }
        }
        grid_barrier(a.barrier, a.error);
        // P: stable scatter into the segment lists; the CSR offsets are the segment starts
        int* const sh_start = mesh_smem;                                                  // [kMaxOnePass]
        uint16_t* const wc = reinterpret_cast<uint16_t*>(mesh_smem + kMaxOnePass);       // [kWarps][kMaxOnePass]
        for (int i = threadIdx.x; i < kWarps * kMaxOnePass / 2; i += kThreads) reinterpret_cast<unsigned*>(wc)[i] = 0u;
        {
            // segment starts: thread t scans its run of kPerT consecutive sizes, loaded together
            constexpr int kPerT = kMaxOnePass / kThreads;
            const int d0 = threadIdx.x * kPerT;
            int v[kPerT];
            int local = 0;
#pragma unroll
            for (int j = 0; j < kPerT; ++j) {
                v[j] = d0 + j < nS ? __ldcg(a.seg_cnt + d0 + j) : 0;
                local += v[j];
            }
            int tot;
            int run = block_exclusive(local, sh_scan, &tot);
#pragma unroll
            for (int j = 0; j < kPerT; ++j) {
                if (d0 + j < nS) {
                    sh_start[d0 + j] = run;
                    if (blockIdx.x == 0) a.seg_offsets[d0 + j] = run;
                }
                run += v[j];
            }
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                a.seg_offsets[nS] = tot;
                a.counts[2] = tot;
            }
        }
        __syncthreads();
        for (int c = blockIdx.x; c < Ct; c += gridDim.x) {
            // warp w owns the 128 consecutive entries [c kChunk + 128 w, + 128), in 4 rounds of 32
            const long long w0 = (long long)c * kChunk + wp * (kChunk / kWarps);
            int rank[kPer], seg[kPer], kk[kPer];
#pragma unroll
            for (int r = 0; r < kPer; ++r) {   // the keys' loads in flight together
                const long long i = w0 + r * 32 + ln;
                kk[r] = i < nT ? __ldcg(a.keys[0] + i) : -1;
            }
#pragma unroll
            for (int r = 0; r < kPer; ++r) {
                int k = kk[r];
                if (k >= nS) k = -1;   // in no segment
                const unsigned peers = __match_any_sync(0xffffffffu, k);
                const unsigned lower = peers & ((1u << ln) - 1u);
                int base = 0;
                if (k >= 0) base = wc[wp * kMaxOnePass + k];
                __syncwarp();
                if (k >= 0 && lower == 0) wc[wp * kMaxOnePass + k] = (uint16_t)(base + __popc(peers));
                __syncwarp();
                rank[r] = base + __popc(lower);
                seg[r] = k;
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < kPer; ++r) {
                const int k = seg[r];
                if (k < 0) continue;
                int pre = 0;   // the segment's entries in the chunk's earlier warps
                for (int w = 0; w < wp; ++w) pre += wc[w * kMaxOnePass + k];
                const long long pos = (long long)sh_start[k] + __ldcg(a.seg_chunk + (long long)k * Ctp + c) + pre + rank[r];
                a.seg_tris[pos] = (int32_t)(w0 + r * 32 + ln);
            }
            __syncthreads();   // every warp has read the counts before any clears its own
#pragma unroll
            for (int r = 0; r < kPer; ++r)
                if (seg[r] >= 0) wc[wp * kMaxOnePass + seg[r]] = 0;
            __syncwarp();
        }
        return;
    }

    // R: stable LSD radix sort of (segment index, T index) over the T entries
    const int key_bits = 32 - __clz(nS);   // keys run over 0..nS
    const int passes = (key_bits + kMaxDigitBits - 1) / kMaxDigitBits;
    const int dbits = (key_bits + passes - 1) / passes;
    const int bins = 1 << dbits;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = dbits * pass;
        const int32_t* ks = a.keys[pass & 1];
        const int32_t* vs = a.vals[pass & 1];
        int32_t* kd = a.keys[(pass + 1) & 1];
        int32_t* vd = a.vals[(pass + 1) & 1];
        // R1: digit histogram of every chunk
        for (int c = blockIdx.x; c < Ct; c += gridDim.x) {
            for (int d = threadIdx.x; d < bins; d += kThreads) sh_bins[d] = 0;
            __syncthreads();
            const long long i0 = (long long)c * kChunk + threadIdx.x * kPer;
#pragma unroll
            for (int j = 0; j < kPer; ++j)
                if (i0 + j < nT) atomicAdd(&sh_bins[(__ldcg(ks + i0 + j) >> shift) & (bins - 1)], 1);
            __syncthreads();
            for (int d = threadIdx.x; d < bins; d += kThreads) a.hist[(long long)d * Ct + c] = sh_bins[d];
            __syncthreads();
        }
        grid_barrier(a.barrier, a.error);
        // R2: per digit, exclusive offsets over the chunks, and the digit's total
        for (int d = blockIdx.x; d < bins; d += gridDim.x) {
            int32_t* h = a.hist + (long long)d * Ct;
            long long carry = 0;
            for (int base = 0; base < Ct; base += kThreads) {
                const int i = base + threadIdx.x;
                const int v = i < Ct ? __ldcg(h + i) : 0;
                int tot;
                const int e = block_exclusive(v, sh_scan, &tot);
                if (i < Ct) h[i] = (int)(carry + e);
                carry += tot;
            }
            if (threadIdx.x == 0) a.bin_tot[d] = (int)carry;
        }
        grid_barrier(a.barrier, a.error);
        // R3: stable scatter
        {
            int tot;
            // the digits' bases: thread t scans its run of consecutive digits
            const int per = (bins + kThreads - 1) / kThreads, d0 = threadIdx.x * per;
            int local = 0;
            for (int d = d0; d < d0 + per && d < bins; ++d) local += __ldcg(a.bin_tot + d);
            int run = block_exclusive(local, sh_scan, &tot);
            for (int d = d0; d < d0 + per && d < bins; ++d) {
                sh_base[d] = run;
                run += __ldcg(a.bin_tot + d);
            }
        }
        for (int c = blockIdx.x; c < Ct; c += gridDim.x) {
            for (int d = threadIdx.x; d < kWarps * bins / 2; d += kThreads) {
                const int w = d / (bins / 2), e = d - w * (bins / 2);
                reinterpret_cast<unsigned*>(sh_wc + w * kMaxBins)[e] = 0u;
            }
            __syncthreads();
            // warp w owns the 256 consecutive entries [c kChunk + 256 w, + 256), in 8 rounds of 32
            const long long w0 = (long long)c * kChunk + warp * (kChunk / kWarps);
            int rank[kPer], dig[kPer];
#pragma unroll
            for (int r = 0; r < kPer; ++r) {
                const long long i = w0 + r * 32 + lane;
                const int d = i < nT ? (__ldcg(ks + i) >> shift) & (bins - 1) : -1;
                const unsigned peers = __match_any_sync(0xffffffffu, d);
                const unsigned lower = peers & ((1u << lane) - 1u);
                int base = 0;
                if (d >= 0) base = sh_wc[warp * kMaxBins + d];
                __syncwarp();
                if (d >= 0 && lower == 0) sh_wc[warp * kMaxBins + d] = (uint16_t)(base + __popc(peers));
                __syncwarp();
                rank[r] = base + __popc(lower);
                dig[r] = d;
            }
            __syncthreads();
            // per digit: offsets of the warps (warp order = entry order)
            for (int d = threadIdx.x; d < bins; d += kThreads) {
                int run = 0;
                for (int w = 0; w < kWarps; ++w) {
                    const int t = sh_wc[w * kMaxBins + d];
                    sh_wc[w * kMaxBins + d] = (uint16_t)run;
                    run += t;
                }
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < kPer; ++r) {
                const int d = dig[r];
                if (d < 0) continue;
                const long long i = w0 + r * 32 + lane;
                const long long pos =
                    (long long)sh_base[d] + __ldcg(a.hist + (long long)d * Ct + c) + sh_wc[warp * kMaxBins + d] + rank[r];
                kd[pos] = __ldcg(ks + i);
                vd[pos] = __ldcg(vs + i);
            }
            __syncthreads();
        }
        grid_barrier(a.barrier, a.error);
    }

    // G: CSR of the segments (their boundary half-edges came with HE in D)
    // keys below nS are the triangles in segments, sorted first
    const int32_t* K = a.keys[passes & 1];
    const int32_t* V = a.vals[passes & 1];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nT; p += stride) {
        const int k = __ldcg(K + p);
        if (k >= nS) continue;
        a.seg_tris[p] = __ldcg(V + p);
        if (p == 0 || __ldcg(K + p - 1) != k) a.seg_offsets[k] = (int32_t)p;
        if (p + 1 == nT || __ldcg(K + p + 1) >= nS) {   // the last triangle in a segment
            a.seg_offsets[nS] = (int32_t)(p + 1);
            a.counts[2] = p + 1;
        }
    }
}

}  // namespace mesh
}  // namespace pl3d

using namespace pl3d;
using namespace pl3d::ctxutil;

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int grow_mesh(pl3d_ctx* c, size_t need, cudaStream_t s) {
    if (c->mslab_cap >= need) return PL3D_OK;
    if (c->mslab && cudaStreamSynchronize(s) != cudaSuccess) return PL3D_ERR_CUDA;
    cudaFree(c->mslab);
    c->mslab = nullptr;
    c->mslab_cap = 0;
    const size_t cap = need + need / 8;
    if (cudaMalloc((void**)&c->mslab, cap) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_OUT_OF_MEMORY;
    }
    c->mslab_cap = cap;
    return PL3D_OK;
}

}  // namespace

extern "C" int pl3d_extract_mesh(pl3d_ctx* ctx, const float* points, const int32_t* labels, int H, int W,
                                 int32_t* out_T, int32_t* out_Tmap, int32_t* out_HE, int64_t* out_counts,
                                 int32_t* out_seg_labels, int32_t* out_seg_offsets, int32_t* out_seg_tris,
                                 uint8_t* out_border, void* stream) {
    if (!ctx || !points || !out_T || !out_Tmap || !out_HE || !out_counts) return PL3D_ERR_INVALID_ARG;
    if (labels && (!out_seg_labels || !out_seg_offsets || !out_seg_tris)) return PL3D_ERR_INVALID_ARG;
    // half-edge ids (3 |T| of them) must fit int32
    if (H < 2 || W < 2 || 6LL * (H - 1) * (long long)(W - 1) >= (1LL << 31) || 3LL * H * W >= (1LL << 31))
        return PL3D_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PL3D_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ntri = 2 * (size_t)(H - 1) * (W - 1);
    const int C = (int)((ntri + mesh::kChunk - 1) / mesh::kChunk);
    // scratch: chunk counts, root index, keys and values (double buffered), histograms,
    // digit totals, flag bits, and the (segment, chunk) counts and segment sizes of the one-pass
    // lists (up to kMaxOnePass segments x C chunks, at most 2^24 entries: 8 B per triangle below
    // that; a frame whose segments need more takes the radix sort)
    const size_t b_cnt = align_up(2 * (size_t)C * 4, 256), b_tri = align_up(ntri * 4, 256);
    const size_t b_hist = align_up((size_t)mesh::kMaxBins * C * 4, 256), b_bins = align_up(mesh::kMaxBins * 4, 256);
    const size_t b_bits = align_up(2 * (size_t)C * (mesh::kChunk / 32) * 4, 256);
    const long long seg_cap = labels ? std::min((long long)mesh::kMaxOnePass * (C + 8), 1LL << 24) : 0;
    const size_t b_segc = align_up((size_t)seg_cap * 4, 256), b_segn = align_up(mesh::kMaxOnePass * 4, 256);
    int rc = grow_mesh(ctx, b_cnt + 5 * b_tri + b_hist + b_bins + b_bits + b_segc + b_segn, s);
    if (rc != PL3D_OK) return rc;
    mesh::MeshArgs a;
    memset(&a, 0, sizeof(a));
    a.points = points;
    a.labels = labels;
    a.H = H;
    a.W = W;
    a.T = out_T;
    a.Tmap = out_Tmap;
    a.HE = out_HE;
    a.counts = reinterpret_cast<long long*>(out_counts);
    a.seg_labels = out_seg_labels;
    a.seg_offsets = out_seg_offsets;
    a.seg_tris = out_seg_tris;
    a.border = out_border;
    a.n_chunks = C;
    unsigned char* p = ctx->mslab;
    a.cnt = reinterpret_cast<int32_t*>(p);
    p += b_cnt;
    a.root_idx = reinterpret_cast<int32_t*>(p);
    p += b_tri;
    for (int i = 0; i < 2; ++i) {
        a.keys[i] = reinterpret_cast<int32_t*>(p);
        p += b_tri;
        a.vals[i] = reinterpret_cast<int32_t*>(p);
        p += b_tri;
    }
    a.hist = reinterpret_cast<int32_t*>(p);
    p += b_hist;
    a.bin_tot = reinterpret_cast<int32_t*>(p);
    p += b_bins;
    a.bits = reinterpret_cast<unsigned*>(p);
    p += b_bits;
    a.seg_chunk = seg_cap > 0 ? reinterpret_cast<int32_t*>(p) : nullptr;
    a.seg_chunk_cap = seg_cap;
    p += b_segc;
    a.seg_cnt = reinterpret_cast<int32_t*>(p);
    a.barrier = ctx->barrier();
    a.error = ctx->error();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PL3D_ERR_CUDA;
    const void* fn = reinterpret_cast<const void*>(&mesh::mesh_kernel);
    // one CTA per chunk (at least one per digit of the radix scans), as many as are resident
    const int want = C > mesh::kMaxBins ? C : mesh::kMaxBins;
    static_assert(mesh::kSmemBytes <= 48 * 1024, "within the default dynamic shared memory: no opt-in per call");
    const int grid = persistent_grid(fn, mesh::kSmemBytes, dev, Tuning{0, 0, 0}, want);
    if (grid <= 0) return PL3D_ERR_CUDA;
    void* args[1] = {&a};
    cudaEvent_t e0, e1;
    record_start(ctx, s, &e0, &e1);
    if (cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kThreads), args, mesh::kSmemBytes, s) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_CUDA;
    }
    record_stop(ctx, s, kSlotMesh, e0, e1);
    ctx->launches += 1;
    return PL3D_OK;
}
