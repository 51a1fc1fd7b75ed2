// Evaluation (outline steps 2-4 of Sec. 3): S2M (P2M), M2M, M2L, S2L (X list), L2L,
// local-expansion and W-list evaluation at the targets, near-field P2P, and the self term.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include <cooperative_groups.h>
#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"
#include "cheb.cuh"
#include "kernel.cuh"

namespace kifmm {

static inline unsigned nbk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------------------------------
// plan-time data for the evaluation
// ------------------------------------------------------------------------------------
__global__ void mark_leaf_points(const int32_t* leaf, const int32_t* pstart, const int32_t* pend,
                                 int64_t nb, int32_t* leaf_of) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb || !leaf[b]) return;
    for (int i = pstart[b]; i < pend[b]; ++i) leaf_of[i] = (int32_t)b;
}

// coordinates relative to the centre of the point's own leaf, rounded once to FP32
__global__ void local_coords(const double* spts, const int32_t* leaf_of, const double* centre,
                             int64_t n, float4* loc) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double* c = centre + 3 * (int64_t)leaf_of[k];
    loc[k] = make_float4((float)(spts[3 * k] - c[0]), (float)(spts[3 * k + 1] - c[1]),
                         (float)(spts[3 * k + 2] - c[2]), 0.f);
}

__global__ void select_boxes(const int32_t* level, const int32_t* leaf, int64_t lo, int64_t hi,
                             int want_leaf, int min_level, int32_t* flag) {
    int64_t b = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= hi) return;
    int f = (level[b] >= min_level) && ((want_leaf < 0) || (leaf[b] == want_leaf));
    flag[b - lo] = f;
}
__global__ void compact_boxes(const int32_t* flag, const int32_t* pos, int64_t lo, int64_t cnt,
                              int32_t* out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt) return;
    if (flag[k]) out[pos[k]] = (int32_t)(lo + k);
}

// (child, parent) pairs for octant o of the non-leaf boxes in [lo, hi)
__global__ void m2m_pairs(const int32_t* child, const int32_t* leaf, int64_t lo, int64_t hi, int o,
                          int32_t* flag) {
    int64_t b = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= hi) return;
    flag[b - lo] = (!leaf[b] && child[8 * b + o] >= 0) ? 1 : 0;
}
__global__ void m2m_fill(const int32_t* child, const int32_t* flag, const int32_t* pos, int64_t lo,
                         int64_t cnt, int o, int32_t* src, int32_t* dst) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt || !flag[k]) return;
    int64_t b = lo + k;
    src[pos[k]] = child[8 * b + o];
    dst[pos[k]] = (int32_t)b;
}


// active offset slots of a tile of boxes (union of their V lists): boxes lo + tile*tb + k,
// or list[tile*tb + k] when a box list is given (k < tb, within the level's hi - lo boxes)
__global__ void m2l_tile_slots(const int32_t* vtab, int64_t lo, int64_t hi, int tb, const int32_t* list,
                               int32_t* slots) {
    int tile = blockIdx.x;
    __shared__ int mask[kOffsetSlots];
    for (int s = threadIdx.x; s < kOffsetSlots; s += blockDim.x) mask[s] = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < tb * kOffsetSlots; e += blockDim.x) {
        int64_t k = (int64_t)tile * tb + e / kOffsetSlots;
        int s = e % kOffsetSlots;
        if (k >= hi - lo) continue;
        int64_t b = list ? list[k] : lo + k;
        if (vtab[b * kOffsetSlots + s] >= 0) mask[s] = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int n = 0;
        for (int s = 0; s < kOffsetSlots; ++s)
            if (mask[s]) slots[(int64_t)tile * kSlotStride + 1 + n++] = s;
        slots[(int64_t)tile * kSlotStride] = n;
    }
}

// V-list entries per level (algorithmic M2L work)
// ptab[b][o] = parent of box b for its octant o inside the parent (boxes of level >= 3), -1 else
__global__ void parent_tab(const int32_t* parent, const int32_t* anchor, const int32_t* level, int64_t nb,
                           int32_t* ptab) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    for (int o = 0; o < 8; ++o) ptab[b * 8 + o] = -1;
    if (level[b] < 3) return;
    const int o = (anchor[3 * b] & 1) | ((anchor[3 * b + 1] & 1) << 1) | ((anchor[3 * b + 2] & 1) << 2);
    ptab[b * 8 + o] = parent[b];
}

// Mc [8][S][R] -> [8][R][R] (rows >= S zero), the square tables of the tensor-core kernel
// Mc [8][S][R] into square tables [8][Mt][Mt] (zero rows i >= S and columns j >= R)
__global__ void pad_mc(const double* Mc, int S, int R, int Mt, double* out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 8LL * Mt * Mt) return;
    const int64_t o = e / ((int64_t)Mt * Mt);
    const int i = (int)((e / Mt) % Mt), j = (int)(e % Mt);
    out[e] = (i < S && j < R) ? Mc[(o * S + i) * R + j] : 0.0;
}

// out[box][j] = (double) in[box][j], j < ncol, for the listed boxes (in rows of R floats)
__global__ void rows_f2d(const int32_t* boxes, int n, const float* in, int R, double* out, int ldo, int ncol) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * ncol) return;
    const int64_t b = boxes[e / ncol];
    const int j = (int)(e % ncol);
    out[b * ldo + j] = (double)in[b * R + j];
}

// L2L slots of a tile: the octants of its boxes (a tile may span two octant groups)
__global__ void l2l_tile_slots(const int4* tiles, int ntiles, const int32_t* boxes, const int32_t* anchor,
                               int32_t* slots) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const int4 tl = tiles[t];
    int mask = 0;
    for (int k = 0; k < tl.z; ++k) {
        const int b = boxes[tl.y + k];
        mask |= 1 << ((anchor[3 * b] & 1) | ((anchor[3 * b + 1] & 1) << 1) | ((anchor[3 * b + 2] & 1) << 2));
    }
    int n = 0;
    for (int o = 0; o < 8; ++o)
        if (mask & (1 << o)) slots[(int64_t)t * kSlotStride + 1 + n++] = o;
    slots[(int64_t)t * kSlotStride] = n;
}

__global__ void count_v_per_level(const int32_t* voff, const int32_t* level, int64_t nb, unsigned long long* cnt) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int n = voff[b + 1] - voff[b];
    if (n > 0) atomicAdd(&cnt[level[b]], (unsigned long long)n);
}

__global__ void kid_table(const int32_t* child, const int32_t* parents, int n, int32_t* kids) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int P = parents[k];
    for (int o = 0; o < 8; ++o) kids[(int64_t)o * n + k] = child[8 * (int64_t)P + o];
}

__global__ void octant_flags(const int32_t* anchor, int64_t lo, int64_t hi, int oc, int32_t* flag) {
    int64_t b = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= hi) return;
    int o = (anchor[3 * b] & 1) | ((anchor[3 * b + 1] & 1) << 1) | ((anchor[3 * b + 2] & 1) << 2);
    flag[b - lo] = (o == oc) ? 1 : 0;
}

__global__ void nonempty_boxes(const int32_t* off, int64_t lo, int64_t hi, int min_level,
                               const int32_t* level, int32_t* flag) {
    int64_t b = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= hi) return;
    flag[b - lo] = (off[b + 1] > off[b] && level[b] >= min_level) ? 1 : 0;
}

constexpr int kM2LTile = 64;     // boxes per M2L tile (both precisions)

// near-field pair evaluations of one evaluation: sum over leaves B of n_B * (sum_{A in U(B)} n_A) - n
__global__ void count_p2p_pairs(const int32_t* leaves, int64_t nl, const int32_t* uoff, const int32_t* uitems,
                                const int32_t* pstart, const int32_t* pend, unsigned long long* out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nl) return;
    int B = leaves[k];
    unsigned long long s = 0;
    for (int u = uoff[B]; u < uoff[B + 1]; ++u) s += (unsigned long long)(pend[uitems[u]] - pstart[uitems[u]]);
    unsigned long long nb = (unsigned long long)(pend[B] - pstart[B]);
    atomicAdd(out, nb * s - nb);
}

static int p2p_series_check(Plan& p);

int build_eval_data(Plan& p) {
    Tree& t = p.tree;
    cudaStream_t st = p.stream;
    const int64_t n = t.n, nb = t.nboxes;
    const int S = p.S;
    // work space of the split SIMT applies: a split launch is at most 4 blocks per SM of at most
    // 64 x 64 FP64 partial sums each
    if (t.nlevels > 2) KF_TRY(dev_alloc(p.apply_part, (size_t)4 * p.num_sms * 64 * 64 * sizeof(double)));
    KF_TRY(dev_alloc(p.leaf_of, n * 4));
    mark_leaf_points<<<nbk(nb, 256), 256, 0, st>>>(ptr<int32_t>(t.leaf), ptr<int32_t>(t.pstart),
                                                    ptr<int32_t>(t.pend), nb, ptr<int32_t>(p.leaf_of));
    KF_LAUNCH();
    KF_TRY(dev_alloc(p.loc32, n * sizeof(float4)));
    local_coords<<<nbk(n, 256), 256, 0, st>>>(ptr<double>(p.pts), ptr<int32_t>(p.leaf_of),
                                              ptr<double>(t.centre), n, ptr<float4>(p.loc32));
    KF_LAUNCH();

    DevBuf flag, pos, scan_tmp;
    KF_TRY(dev_alloc(flag, (nb + 1) * 4));
    KF_TRY(dev_alloc(pos, (nb + 1) * 4));
    // all leaves, and leaves of level >= 2 (P2M)
    {
        select_boxes<<<nbk(nb, 256), 256, 0, st>>>(ptr<int32_t>(t.level), ptr<int32_t>(t.leaf), 0, nb, 1, 0,
                                                   ptr<int32_t>(flag));
        KF_LAUNCH();
        int32_t tot = 0;
        KF_TRY(device_scan_i32(ptr<int32_t>(flag), ptr<int32_t>(pos), nb, &tot, st, scan_tmp));
        KF_TRY(dev_alloc(p.leaves, (size_t)std::max(tot, 1) * 4));
        compact_boxes<<<nbk(nb, 256), 256, 0, st>>>(ptr<int32_t>(flag), ptr<int32_t>(pos), 0, nb,
                                                     ptr<int32_t>(p.leaves));
        KF_LAUNCH();
        p.nleaves = tot;
        select_boxes<<<nbk(nb, 256), 256, 0, st>>>(ptr<int32_t>(t.level), ptr<int32_t>(t.leaf), 0, nb, 1, 2,
                                                   ptr<int32_t>(flag));
        KF_LAUNCH();
        KF_TRY(device_scan_i32(ptr<int32_t>(flag), ptr<int32_t>(pos), nb, &tot, st, scan_tmp));
        KF_TRY(dev_alloc(p.p2m_boxes, (size_t)std::max(tot, 1) * 4));
        compact_boxes<<<nbk(nb, 256), 256, 0, st>>>(ptr<int32_t>(flag), ptr<int32_t>(pos), 0, nb,
                                                     ptr<int32_t>(p.p2m_boxes));
        KF_LAUNCH();
        p.n_p2m = tot;
        // leaves with a non-empty W list
        nonempty_boxes<<<nbk(nb, 256), 256, 0, st>>>(ptr<int32_t>(p.lists[2].off), 0, nb, 0,
                                                     ptr<int32_t>(t.level), ptr<int32_t>(flag));
        KF_LAUNCH();
        KF_TRY(device_scan_i32(ptr<int32_t>(flag), ptr<int32_t>(pos), nb, &tot, st, scan_tmp));
        KF_TRY(dev_alloc(p.wleaves, (size_t)std::max(tot, 1) * 4));
        compact_boxes<<<nbk(nb, 256), 256, 0, st>>>(ptr<int32_t>(flag), ptr<int32_t>(pos), 0, nb,
                                                     ptr<int32_t>(p.wleaves));
        KF_LAUNCH();
        p.n_wleaves = tot;
    }
    {
        DevBuf cnt;
        KF_TRY(dev_alloc(cnt, 8));
        KF_CUDA(cudaMemsetAsync(cnt.p, 0, 8, st));
        if (p.nleaves > 0) {
            count_p2p_pairs<<<nbk(p.nleaves, 256), 256, 0, st>>>(ptr<int32_t>(p.leaves), p.nleaves,
                                                                 ptr<int32_t>(p.lists[0].off), ptr<int32_t>(p.lists[0].items),
                                                                 ptr<int32_t>(t.pstart), ptr<int32_t>(t.pend),
                                                                 ptr<unsigned long long>(cnt));
            KF_LAUNCH();
        }
        unsigned long long h = 0;
        KF_CUDA(cudaMemcpyAsync(&h, cnt.p, 8, cudaMemcpyDeviceToHost, st));
        KF_CUDA(cudaStreamSynchronize(st));
        p.p2p_pairs = (int64_t)h;
        dev_free(cnt);
    }
    {   // algorithmic work of one evaluation: M2L 2 r_l^2 per V pair; FP64 upward 2 r_l S per
        // leaf (projection) and 2 r_l r_{l+1} per child (M2M)
        DevBuf cnt;
        KF_TRY(dev_alloc(cnt, 32 * 8));
        KF_CUDA(cudaMemsetAsync(cnt.p, 0, 32 * 8, st));
        count_v_per_level<<<nbk(nb, 256), 256, 0, st>>>(ptr<int32_t>(p.lists[1].off), ptr<int32_t>(t.level), nb,
                                                         ptr<unsigned long long>(cnt));
        KF_LAUNCH();
        unsigned long long hc[32];
        KF_CUDA(cudaMemcpyAsync(hc, cnt.p, 32 * 8, cudaMemcpyDeviceToHost, st));
        KF_CUDA(cudaStreamSynchronize(st));
        dev_free(cnt);
        p.m2l_flops = 0;
        for (int l = 2; l < t.nlevels; ++l) p.m2l_flops += 2.0 * p.ops[l].rank * p.ops[l].rank * (double)hc[l];
    }
    p.lv.clear();
    p.lv.resize(t.nlevels);
    for (int l = 2; l < t.nlevels; ++l) {
        auto& L = p.lv[l];
        int64_t lo = t.level_start[l], hi = t.level_start[l + 1], cnt = hi - lo;
        L.n_all = (int)cnt;
        // M2M pairs per octant (parents at level l, children at l + 1)
        for (int o = 0; o < 8; ++o) {
            m2m_pairs<<<nbk(cnt, 256), 256, 0, st>>>(ptr<int32_t>(t.child), ptr<int32_t>(t.leaf), lo, hi, o,
                                                     ptr<int32_t>(flag));
            KF_LAUNCH();
            int32_t tot = 0;
            KF_TRY(device_scan_i32(ptr<int32_t>(flag), ptr<int32_t>(pos), cnt, &tot, st, scan_tmp));
            KF_TRY(dev_alloc(L.m2m_src[o], (size_t)std::max(tot, 1) * 4));
            KF_TRY(dev_alloc(L.m2m_dst[o], (size_t)std::max(tot, 1) * 4));
            m2m_fill<<<nbk(cnt, 256), 256, 0, st>>>(ptr<int32_t>(t.child), ptr<int32_t>(flag), ptr<int32_t>(pos),
                                                    lo, cnt, o, ptr<int32_t>(L.m2m_src[o]),
                                                    ptr<int32_t>(L.m2m_dst[o]));
            KF_LAUNCH();
            L.n_m2m[o] = tot;
        }
        {   // the same pairs concatenated over the octants, for the batched L2L launch
            int32_t hoff[9] = {0};
            for (int o = 0; o < 8; ++o) hoff[o + 1] = hoff[o] + L.n_m2m[o];
            KF_TRY(dev_alloc(L.l2l_src, (size_t)std::max(hoff[8], 1) * 4));
            KF_TRY(dev_alloc(L.l2l_dst, (size_t)std::max(hoff[8], 1) * 4));
            KF_TRY(dev_alloc(L.l2l_off, 9 * 4));
            L.l2l_max = 0;
            for (int o = 0; o < 8; ++o) {
                if (L.n_m2m[o] == 0) continue;
                KF_CUDA(cudaMemcpyAsync(ptr<int32_t>(L.l2l_src) + hoff[o], L.m2m_dst[o].p, L.n_m2m[o] * 4,
                                        cudaMemcpyDeviceToDevice, st));   // parents
                KF_CUDA(cudaMemcpyAsync(ptr<int32_t>(L.l2l_dst) + hoff[o], L.m2m_src[o].p, L.n_m2m[o] * 4,
                                        cudaMemcpyDeviceToDevice, st));   // children
                L.l2l_max = std::max(L.l2l_max, L.n_m2m[o]);
            }
            KF_CUDA(cudaMemcpyAsync(L.l2l_off.p, hoff, 9 * 4, cudaMemcpyHostToDevice, st));
            KF_CUDA(cudaStreamSynchronize(st));
        }
        // M2L tiles and their active offset slots
        int tb = kM2LTile;
        L.n_tiles = (int)((cnt + tb - 1) / tb);
        KF_TRY(dev_alloc(L.m2l_slots, (size_t)std::max(L.n_tiles, 1) * kSlotStride * 4));
        if (L.n_tiles > 0) {
            m2l_tile_slots<<<L.n_tiles, 256, 0, st>>>(ptr<int32_t>(p.vtab), lo, hi, tb, nullptr, ptr<int32_t>(L.m2l_slots));
            KF_LAUNCH();
        }
        // non-leaf boxes of this level and their children per octant (-1: empty octant)
        select_boxes<<<nbk(cnt, 256), 256, 0, st>>>(ptr<int32_t>(t.level), ptr<int32_t>(t.leaf), lo, hi, 0, 2,
                                                    ptr<int32_t>(flag) + lo);
        KF_LAUNCH();
        {
            int32_t npar = 0;
            KF_TRY(device_scan_i32(ptr<int32_t>(flag) + lo, ptr<int32_t>(pos), cnt, &npar, st, scan_tmp));
            KF_TRY(dev_alloc(L.parents, (size_t)std::max(npar, 1) * 4));
            KF_TRY(dev_alloc(L.par_kids, (size_t)std::max(npar, 1) * 8 * 4));
            compact_boxes<<<nbk(cnt, 256), 256, 0, st>>>(ptr<int32_t>(flag) + lo, ptr<int32_t>(pos), lo, cnt,
                                                          ptr<int32_t>(L.parents));
            KF_LAUNCH();
            if (npar > 0) {
                kid_table<<<nbk(npar, 256), 256, 0, st>>>(ptr<int32_t>(t.child), ptr<int32_t>(L.parents), npar,
                                                          ptr<int32_t>(L.par_kids));
                KF_LAUNCH();
            }
            L.n_par = npar;
        }
        // leaves of this level
        select_boxes<<<nbk(cnt, 256), 256, 0, st>>>(ptr<int32_t>(t.level), ptr<int32_t>(t.leaf), lo, hi, 1, 2,
                                                    ptr<int32_t>(flag) + lo);
        KF_LAUNCH();
        {
            int32_t nlf = 0;
            KF_TRY(device_scan_i32(ptr<int32_t>(flag) + lo, ptr<int32_t>(pos), cnt, &nlf, st, scan_tmp));
            KF_TRY(dev_alloc(L.leafs, (size_t)std::max(nlf, 1) * 4));
            compact_boxes<<<nbk(cnt, 256), 256, 0, st>>>(ptr<int32_t>(flag) + lo, ptr<int32_t>(pos), lo, cnt,
                                                          ptr<int32_t>(L.leafs));
            KF_LAUNCH();
            L.n_leaf = nlf;
        }
        // upward solves of the level: its leaves, then its parents
        L.n_up = L.n_leaf + L.n_par;
        KF_TRY(dev_alloc(L.upb, (size_t)std::max(L.n_up, 1) * 4));
        if (L.n_leaf > 0)
            KF_CUDA(cudaMemcpyAsync(L.upb.p, L.leafs.p, (size_t)L.n_leaf * 4, cudaMemcpyDeviceToDevice, st));
        if (L.n_par > 0)
            KF_CUDA(cudaMemcpyAsync(ptr<int32_t>(L.upb) + L.n_leaf, L.parents.p, (size_t)L.n_par * 4,
                                    cudaMemcpyDeviceToDevice, st));
        // boxes with a non-empty X list
        nonempty_boxes<<<nbk(cnt, 256), 256, 0, st>>>(ptr<int32_t>(p.lists[3].off), lo, hi, 2,
                                                       ptr<int32_t>(t.level), ptr<int32_t>(flag));
        KF_LAUNCH();
        int32_t tot = 0;
        KF_TRY(device_scan_i32(ptr<int32_t>(flag), ptr<int32_t>(pos), cnt, &tot, st, scan_tmp));
        KF_TRY(dev_alloc(L.xboxes, (size_t)std::max(tot, 1) * 4));
        compact_boxes<<<nbk(cnt, 256), 256, 0, st>>>(ptr<int32_t>(flag), ptr<int32_t>(pos), lo, cnt,
                                                      ptr<int32_t>(L.xboxes));
        KF_LAUNCH();
        L.n_x = tot;
    }
    // tensor-core M2L: tiles of 128 boxes over all levels, deepest level first; within a
    // level the boxes are grouped by their octant inside the parent (one set of offsets)
    if (p.m2l_tensor) {
        int64_t nbx = 0;
        int ntiles = 0;
        for (int l = 2; l < t.nlevels; ++l) {
            int64_t c = t.level_start[l + 1] - t.level_start[l];
            nbx += c;
            ntiles += (int)((c + 127) / 128);
        }
        KF_TRY(dev_alloc(p.tc_boxes, (size_t)std::max<int64_t>(nbx, 1) * 4));
        KF_TRY(dev_alloc(p.tc_slots, (size_t)std::max(ntiles, 1) * kSlotStride * 4));
        KF_TRY(dev_alloc(p.tc_tiles, (size_t)std::max(ntiles, 1) * sizeof(int4)));
        std::vector<int4> tiles;
        int64_t off = 0;
        for (int l = t.nlevels - 1; l >= 2; --l) {
            const int64_t lo = t.level_start[l], hi = t.level_start[l + 1], cnt = hi - lo;
            if (cnt <= 0) continue;
            int32_t done = 0;
            for (int oc = 0; oc < 8; ++oc) {
                octant_flags<<<nbk(cnt, 256), 256, 0, st>>>(ptr<int32_t>(t.anchor), lo, hi, oc, ptr<int32_t>(flag));
                KF_LAUNCH();
                int32_t nsel = 0;
                KF_TRY(device_scan_i32(ptr<int32_t>(flag), ptr<int32_t>(pos), cnt, &nsel, st, scan_tmp));
                compact_boxes<<<nbk(cnt, 256), 256, 0, st>>>(ptr<int32_t>(flag), ptr<int32_t>(pos), lo, cnt,
                                                              ptr<int32_t>(p.tc_boxes) + off + done);
                KF_LAUNCH();
                done += nsel;
            }
            const int nt = (int)((cnt + 127) / 128);
            m2l_tile_slots<<<nt, 256, 0, st>>>(ptr<int32_t>(p.vtab), lo, hi, 128, ptr<int32_t>(p.tc_boxes) + off,
                                               ptr<int32_t>(p.tc_slots) + (int64_t)tiles.size() * kSlotStride);
            KF_LAUNCH();
            p.tc_first[l] = (int)tiles.size();
            p.tc_count[l] = nt;
            for (int k = 0; k < nt; ++k)
                tiles.push_back(make_int4(l, (int)(off + 128 * k), (int)std::min<int64_t>(128, cnt - 128 * k), 0));
            off += cnt;
        }
        p.tc_ntiles = (int)tiles.size();
        if (!tiles.empty())
            KF_CUDA(cudaMemcpyAsync(p.tc_tiles.p, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
        // L2L through the same kernel: per child tile the parent at its octant's slot, the
        // parent level's L2L matrices as FP16 hi / lo tables (KIFMM_L2L=simt keeps the SIMT apply)
        const char* l2l = std::getenv("KIFMM_L2L");
        p.l2l_tc = !(l2l && std::string(l2l) == "simt") && t.nlevels > 3 && !tiles.empty();
        if (p.l2l_tc) {
            KF_TRY(dev_alloc(p.ptab, (size_t)nb * 8 * 4));
            parent_tab<<<nbk(nb, 256), 256, 0, st>>>(ptr<int32_t>(t.parent), ptr<int32_t>(t.anchor),
                                                      ptr<int32_t>(t.level), nb, ptr<int32_t>(p.ptab));
            KF_LAUNCH();
            KF_TRY(dev_alloc(p.l2l_slots, tiles.size() * kSlotStride * 4));
            l2l_tile_slots<<<nbk((int64_t)tiles.size(), 128), 128, 0, st>>>(ptr<int4>(p.tc_tiles), (int)tiles.size(),
                                                                            ptr<int32_t>(p.tc_boxes),
                                                                            ptr<int32_t>(t.anchor),
                                                                            ptr<int32_t>(p.l2l_slots));
            KF_LAUNCH();
            for (int l = 2; l + 1 < t.nlevels; ++l) {
                LevelOps& op = p.ops[l];
                KF_TRY(dev_alloc(op.Lhi, (size_t)m2l_tc_table_elems(p.R, 8) * 2));
                KF_TRY(dev_alloc(op.Llo, (size_t)m2l_tc_table_elems(p.R, 8) * 2));
                KF_TRY(m2l_tc_prepare(st, ptr<double>(op.Lo), p.R, op.Lhi.p, op.Llo.p, &op.l2l_sT, 8));
            }
        }
        // M2M translations likewise: per parent tile the 8 child octants as slots (the tree's child
        // table is the source table), Mc padded to square tables of Mt = max(S, R) rounded to 32,
        // the result staged in FP32 and copied into the parents' check rows (KIFMM_M2M=simt keeps
        // the FP32 M2M kernels). By default only when S <= R: with more check points than coefficients
        // (S > R) the children's c pass through FP16 hi / lo rows padded to Mt, whose 22 bits
        // relative to each row's largest value cost 1.5e-7 of the mixed form's error at 7.6 Torr
        // (1.03e-6 against 8.9e-7 with the FP32 apply), beyond the 1e-6 gate; KIFMM_M2M=tc takes
        // the tensor cores there too. Surface form only: the Chebyshev translations (K = p^3 = 512
        // at p = 8) would take 96 truncating accumulations per slot, a bias that compounds level by
        // level up the tree.
        const char* m2m = std::getenv("KIFMM_M2M");
        p.m2m_R = (std::max(S, p.R) + 31) / 32 * 32;
        const bool m2m_force = m2m && std::string(m2m) == "tc";
        p.m2m_tc = !(m2m && std::string(m2m) == "simt") && t.nlevels > 3 && !p.cheb && m2l_tc_supported(p.m2m_R) &&
                   (S <= p.R || m2m_force);
        if (p.m2m_tc) {
            const int R = p.m2m_R;
            std::vector<int4> mt;
            DevBuf pad;
            KF_TRY(dev_alloc(pad, (size_t)8 * R * R * 8));
            for (int l = 2; l + 1 < t.nlevels; ++l) {
                LevelOps& op = p.ops[l];
                p.m2m_first[l] = (int)mt.size();
                const int np = p.lv[l].n_par;
                p.m2m_count[l] = (np + 127) / 128;
                for (int k = 0; k < p.m2m_count[l]; ++k) mt.push_back(make_int4(l, 128 * k, std::min(128, np - 128 * k), 0));
                if (np == 0) continue;
                pad_mc<<<nbk(8LL * R * R, 256), 256, 0, st>>>(ptr<double>(op.Mc), S, p.R, R, ptr<double>(pad));
                KF_LAUNCH();
                KF_TRY(dev_alloc(op.Mhi, (size_t)m2l_tc_table_elems(R, 8) * 2));
                KF_TRY(dev_alloc(op.Mlo, (size_t)m2l_tc_table_elems(R, 8) * 2));
                KF_TRY(m2l_tc_prepare(st, ptr<double>(pad), R, op.Mhi.p, op.Mlo.p, &op.m2m_sT, 8));
            }
            dev_free(pad);
            std::vector<int32_t> ms(std::max<size_t>(mt.size(), 1) * kSlotStride, 0);
            for (size_t k = 0; k < mt.size(); ++k) {
                ms[k * kSlotStride] = 8;
                for (int o = 0; o < 8; ++o) ms[k * kSlotStride + 1 + o] = o;
            }
            KF_TRY(dev_alloc(p.m2m_tiles, std::max<size_t>(mt.size(), 1) * sizeof(int4)));
            KF_TRY(dev_alloc(p.m2m_slots, ms.size() * 4));
            KF_TRY(dev_alloc(p.stage32, (size_t)nb * R * 4));
            if (R > p.R) {
                KF_TRY(dev_alloc(p.m2m_hi, (size_t)nb * R * 2));
                KF_TRY(dev_alloc(p.m2m_lo, (size_t)nb * R * 2));
            }
            if (!mt.empty())
                KF_CUDA(cudaMemcpyAsync(p.m2m_tiles.p, mt.data(), mt.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
            KF_CUDA(cudaMemcpyAsync(p.m2m_slots.p, ms.data(), ms.size() * 4, cudaMemcpyHostToDevice, st));
        }
        KF_CUDA(cudaStreamSynchronize(st));
    }
    // workspace
    const int R = p.R;
    const size_t ts = p.precision == KIFMM_MIXED ? 4 : 8;
    KF_TRY(dev_alloc(p.q, n * 8));
    KF_TRY(dev_alloc(p.Isort, n * 8));
    KF_TRY(dev_alloc(p.far, n * 8));
    KF_TRY(dev_alloc(p.chk, (size_t)nb * S * 8));
    KF_TRY(dev_alloc(p.cu, (size_t)nb * R * 8));
    KF_TRY(dev_alloc(p.dd, (size_t)nb * R * ts));
    if (!p.cheb) {   // the Chebyshev representation reads the node values d and c in place
        KF_TRY(dev_alloc(p.phid, (size_t)nb * S * ts));
        KF_CUDA(cudaMemsetAsync(p.phid.p, 0, (size_t)nb * S * ts, st));
    }
    if (p.precision == KIFMM_MIXED) KF_TRY(dev_alloc(p.cu32, (size_t)nb * R * 4));
    if (p.m2l_tensor) {
        KF_TRY(dev_alloc(p.chi, (size_t)nb * R * 2));
        KF_TRY(dev_alloc(p.clo, (size_t)nb * R * 2));
        KF_TRY(dev_alloc(p.cexp, (size_t)nb * 4));
    }
    if (p.lists[3].len > 0 && !p.cheb) KF_TRY(dev_alloc(p.chkx, (size_t)nb * S * ts));
    if (p.lists[2].len > 0 && !p.cheb) {
        KF_TRY(dev_alloc(p.phiu, (size_t)nb * S * ts));
        KF_CUDA(cudaMemsetAsync(p.phiu.p, 0, (size_t)nb * S * ts, st));
    }
    KF_CUDA(cudaStreamSynchronize(st));
    dev_free(flag); dev_free(pos); dev_free(scan_tmp);
    if (p.precision == KIFMM_MIXED) KF_TRY(p2p_series_check(p));
    KF_TRY(near_tc_plan(p));
    // FP64-exact upward solves on the tensor cores (mixed form; KIFMM_UPWARD=fp64 keeps the FP64 pipe)
    {
        const char* up = std::getenv("KIFMM_UPWARD");
        p.oz = p.precision == KIFMM_MIXED && !p.cheb && pinv_oz_supported(S) && !(up && std::string(up) == "fp64");
        const char* om = std::getenv("KIFMM_OZ_MIN");   // level-size threshold (tests use 0)
        p.oz_min = om ? std::max(0, std::atoi(om)) : kOzMinBoxes;
        // smallest tile count of a level whose M2M / L2L take the tensor-core translation
        // kernel (tests use 1, so that small trees run every tensor-core path)
        const char* tm = std::getenv("KIFMM_TC_MIN_TILES");
        p.tc_min_tiles = tm ? std::max(1, std::atoi(tm)) : kTcMinTiles;
    }
    if (p.oz) {
        int nmax = 0;
        for (int l = 2; l < t.nlevels; ++l) {
            LevelOps& op = p.ops[l];
            if (p.lv[l].n_up == 0) continue;
            nmax = std::max(nmax, p.lv[l].n_up);
            KF_TRY(dev_alloc(op.ozG1, pinv_oz_op_bytes(S, op.rank)));
            KF_TRY(dev_alloc(op.ozEr, (size_t)((op.rank + 47) / 48 * 48) * 4));
            KF_TRY(pinv_oz_prepare(st, ptr<double>(op.G1), S, op.rank, op.ozG1.p, ptr<int>(op.ozEr)));
        }
        KF_TRY(dev_alloc(p.ozBox, std::max<size_t>(pinv_oz_box_bytes(S, nmax), 16)));
        KF_TRY(dev_alloc(p.ozEb, (size_t)std::max(nmax + 128, 1) * 4));
        KF_CUDA(cudaStreamSynchronize(st));
    }
    KF_TRY(lat_up_plan(p));
    return KIFMM_OK;
}

// ------------------------------------------------------------------------------------
// evaluation kernels
// ------------------------------------------------------------------------------------
struct EvalView {
    const double* pts;      // sorted coordinates
    const float4* loc;      // coordinates relative to own leaf centre (FP32)
    const double* centre;   // box centres
    const int32_t* level;
    const int32_t* pstart;
    const int32_t* pend;
    const double* surf;     // unit lattice (3*S); Chebyshev representation: the unit nodes
    double side;
    int S;
    KParams kp;
    double rf_dchk;         // radius of the downward check surface in half-widths (Chebyshev: 1)
    double rf_ueq;          // radius of the upward equivalent surface in half-widths (Chebyshev: 1)
    double rf_out;          // radius of the upward check / downward equivalent surface (surface form)
    int ldu;                // row stride of the upward densities read by the W list
    int cheb;               // Chebyshev representation: the local part of L2P is interpolation
    int cp;                 // Chebyshev order p
    const double* ctab;     // Chebyshev weight table c_k T_k(xbar_n), row stride kChebTab
    const float* ctab32;
    int64_t n_real;         // the caller's points (sorted points with perm >= n_real are padding cells)
};

__device__ __forceinline__ double half_width(const EvalView& E, int lev) {
    return E.side / (double)(2ll << lev);
}

template <class T>
__global__ void k_scatter_q(const T* I, const int32_t* perm, const double* w, int64_t n, int64_t n_real, double* Is,
                            double* q) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t j = perm[k];
    const double v = j < n_real ? (double)I[j] : 0.0;   // padding cells: I = 0
    Is[k] = v;
    q[k] = v * w[k];
}


// S2M (Eq. (s2m), first step): upward check potential of a leaf from its own sources.
// One block per leaf; check points x_j = c_B + r_out r s_j, sources relative to c_B.
constexpr int P2M_T = 160;
// FP32 kernel without the series branch: valid where (b - a) R >= 0.5 for every pair
__device__ __forceinline__ float kern_plain_f32(float r2, const KParams& k) {
    const float rinv = rsqrt_approx(r2);
    const float R = r2 * rinv;
    return (ex2_approx(-k.a_l2e * R) - ex2_approx(-k.b_l2e * R)) * k.norm_f * (rinv * (rinv * rinv));
}
// SER: some source of a leaf may lie closer than 0.5 / (b - a) to its check surface
template <bool MIXED, bool SER>
__global__ void __launch_bounds__(P2M_T) k_p2m(EvalView E, const int32_t* boxes, const double* q, double* chk) {
    const int B = boxes[blockIdx.x];
    const int S = E.S;
    const double r = half_width(E, E.level[B]);
    const int p0 = E.pstart[B], p1 = E.pend[B];
    __shared__ float4 sp32[256];
    __shared__ double sp64[256][4];
    const double* c = E.centre + 3 * (int64_t)B;
    for (int j0 = 0; j0 < S; j0 += P2M_T) {
        const int j = j0 + threadIdx.x;
        double xj[3];
        for (int k = 0; k < 3; ++k) xj[k] = E.rf_out * r * E.surf[3 * min(j, S - 1) + k];
        Kahan acc32;
        double acc64 = 0;
        for (int s0 = p0; s0 < p1; s0 += 256) {
            const int ns = min(256, p1 - s0);
            __syncthreads();
            for (int e = threadIdx.x; e < ns; e += P2M_T) {
                if (MIXED) {
                    float4 v = E.loc[s0 + e];
                    v.w = (float)q[s0 + e];
                    sp32[e] = v;
                } else {
                    for (int k = 0; k < 3; ++k) sp64[e][k] = E.pts[3 * (int64_t)(s0 + e) + k] - c[k];
                    sp64[e][3] = q[s0 + e];
                }
            }
            __syncthreads();
            if (MIXED) {
                const float x0 = (float)xj[0], x1 = (float)xj[1], x2 = (float)xj[2];
                int e = 0;
                for (; e + 7 < ns; e += 8) {   // plain FP32 sums of 8 terms, compensated across blocks
                    float part = 0.f;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const float4 v = sp32[e + u];
                        const float dx = x0 - v.x, dy = x1 - v.y, dz = x2 - v.z;
                        const float r2 = dx * dx + dy * dy + dz * dz;
                        part = fmaf(SER ? kern_f32(r2, E.kp) : kern_plain_f32(r2, E.kp), v.w, part);
                    }
                    acc32.add(part);
                }
                for (; e < ns; ++e) {
                    const float4 v = sp32[e];
                    const float dx = x0 - v.x, dy = x1 - v.y, dz = x2 - v.z;
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    acc32.add((SER ? kern_f32(r2, E.kp) : kern_plain_f32(r2, E.kp)) * v.w);
                }
            } else {
                for (int e = 0; e < ns; ++e) {
                    const double dx = xj[0] - sp64[e][0], dy = xj[1] - sp64[e][1], dz = xj[2] - sp64[e][2];
                    acc64 += kern_f64(sqrt(dx * dx + dy * dy + dz * dz), E.kp) * sp64[e][3];
                }
            }
        }
        if (j < S) chk[(int64_t)B * S + j] = MIXED ? acc32.value() : acc64;
    }
}

// out[dst(c)][row] (+)= sum_t sum_k Op_t[row][k] * in[src_t(c)][k] for row < Mo, k < Ki,
// c < count: translation matrices applied to many boxes (a GEMM whose columns are gathered
// and scattered by box index). Op_t = Op + t * op_stride (row stride ldop), t < nterm;
// src_t(c) = src[t * count + c] (-1: no term), or base + c when src is NULL; dst NULL means
// base + c. Tile TM = 16*RM rows x TN = 16*CN boxes, k-chunks of 16; each thread RM x CN.
// Arithmetic in T; the input is read as TI and the output stored as TO.
constexpr int AP_TK = 16;
constexpr int AP_NT = 8;   // terms whose source indices a block stages in shared memory
// With zoff != NULL the launch is a batch over blockIdx.z: batch z uses Op + z * zstride and
// the columns [zoff[z], zoff[z+1]) of src/dst (count is then the largest batch). With
// zoff == NULL and gridDim.z > 1 the work items (term, k-chunk), taken term-major, are split
// into gridDim.z contiguous ranges: each range's partial sums go to part[z][col][row]
// (col < gridDim.x TN, row < gridDim.y TM) and k_apply_finish adds them in z order, so the
// result does not depend on the order in which blocks finish (without part they are added
// atomically into out, which the caller zeroes). The next item's operands are loaded into
// registers while the current one is multiplied.
template <class T, class TI, class TO, int RM, int CN>
__global__ void __launch_bounds__(256) k_apply(const T* __restrict__ Op, int64_t op_stride, int ldop, int nterm,
                                               int Mo, int Ki, const int32_t* src, const int32_t* dst, int64_t base,
                                               int count, const TI* __restrict__ in, int ldi, TO* out, int ldo,
                                               int accumulate, const int32_t* zoff, int64_t zstride, TO* part) {
    constexpr int TM = 16 * RM, TN = 16 * CN;
    const int nkc = (Ki + AP_TK - 1) / AP_TK;
    int it0 = 0, it1 = nterm * nkc;
    const bool split = !zoff && gridDim.z > 1;
    if (zoff) {
        const int z = blockIdx.z;
        Op += (int64_t)z * zstride;
        src += zoff[z];
        dst += zoff[z];
        count = zoff[z + 1] - zoff[z];
        if ((int)(blockIdx.x * TN) >= count) return;
    } else if (split) {
        const int per = (it1 + gridDim.z - 1) / gridDim.z;
        it0 = min(it1, (int)blockIdx.z * per);
        it1 = min(it1, it0 + per);
    }
    __shared__ T As[AP_TK][TM + 1];
    __shared__ T Bs[AP_TK][TN + 1];
    __shared__ int32_t sidx[AP_NT][TN];   // the block's source boxes per term (nterm <= AP_NT)
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int row0 = blockIdx.y * TM, col0 = blockIdx.x * TN;
    const bool staged = src && nterm <= AP_NT;
    if (staged) {   // one dependent global load per gathered value instead of two
        for (int e = tid; e < nterm * TN; e += 256) {
            const int t = e / TN, col = col0 + e % TN;
            sidx[t][e % TN] = col < count ? src[(int64_t)t * count + col] : -1;
        }
        __syncthreads();
    }
    T acc[RM][CN] = {};
    T ra[RM], rb[CN];
    auto load = [&](int it) {
        const int t = it / nkc, k0 = (it % nkc) * AP_TK;
        const T* Opt = Op + (int64_t)t * op_stride;
#pragma unroll
        for (int i = 0; i < RM; ++i) {
            const int e = tid + 256 * i;
            const int row = row0 + e / AP_TK, k = k0 + e % AP_TK;
            ra[i] = (row < Mo && k < Ki) ? Opt[(int64_t)row * ldop + k] : T(0);
        }
#pragma unroll
        for (int j = 0; j < CN; ++j) {
            const int e = tid + 256 * j;
            const int col = col0 + e / AP_TK, k = k0 + e % AP_TK;
            T v = T(0);
            if (col < count && k < Ki) {
                const int64_t b = staged ? (int64_t)sidx[t][col - col0]
                                  : src ? (int64_t)src[(int64_t)t * count + col] : base + col;
                if (b >= 0) v = (T)in[b * ldi + k];
            }
            rb[j] = v;
        }
    };
    if (it0 < it1) load(it0);
    for (int it = it0; it < it1; ++it) {
#pragma unroll
        for (int i = 0; i < RM; ++i) {
            const int e = tid + 256 * i;
            As[e % AP_TK][e / AP_TK] = ra[i];
        }
#pragma unroll
        for (int j = 0; j < CN; ++j) {
            const int e = tid + 256 * j;
            Bs[e % AP_TK][e / AP_TK] = rb[j];
        }
        __syncthreads();
        if (it + 1 < it1) load(it + 1);
#pragma unroll
        for (int kk = 0; kk < AP_TK; ++kk) {
            T av[RM], bv[CN];
#pragma unroll
            for (int i = 0; i < RM; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < CN; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < CN; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < RM; ++i) {
        int row = row0 + ty + 16 * i;
        if (row >= Mo) continue;
#pragma unroll
        for (int j = 0; j < CN; ++j) {
            int col = col0 + tx + 16 * j;
            if (col >= count) continue;
            int64_t b = dst ? dst[col] : base + col;
            TO* o = out + b * ldo + row;
            if (split && part) part[((int64_t)blockIdx.z * gridDim.x * TN + col) * (gridDim.y * TM) + row] = (TO)acc[i][j];
            else if (split) atomicAdd(o, (TO)acc[i][j]);
            else *o = accumulate ? *o + (TO)acc[i][j] : (TO)acc[i][j];
        }
    }
}
// out[dst(col)][row] (+)= sum over z of part[z][col][row], z in order, a thread per output
// (consecutive threads read consecutive rows of each partial)
template <class TO>
__global__ void k_apply_finish(const TO* __restrict__ part, int nz, int64_t ncp, int nrp, int count, int Mo,
                                 const int32_t* dst, int64_t base, TO* out, int ldo, int accumulate) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)count * Mo) return;
    const int64_t col = e / Mo;
    const int row = (int)(e - col * Mo);
    TO sum = 0;
    for (int z = 0; z < nz; ++z) sum += part[((int64_t)z * ncp + col) * nrp + row];
    const int64_t b = dst ? dst[col] : base + col;
    TO* o = out + b * ldo + row;
    *o = accumulate ? *o + sum : sum;
}

// FP32 translations of the mixed surface form on the SIMT pipes, for at most 160 output rows
// and input ranks K <= 128: a block takes one operator (one octant) and TN coefficient rows,
// and a thread holds 4 output rows rq + 40 i x 4 coefficient rows pq + TN/4 j. The block
// copies all its K / 32 operator chunks into shared memory at once (asynchronous 16-byte
// copies) and loads (and rounds) the coefficient chunks into registers beside them, so it
// waits for memory once; both operands are stored along k (float4 reads, conflict-free).
// Operators are [8][rows][ld] with ld a multiple of 32, so each chunk's operator rows lie
// inside them; columns past K multiply zeros.
constexpr int MM_TK = 32, MM_TM = 160, MM_NS = 4, MM_LD = MM_TK + 4, MM_LDP = MM_TM + 4;
template <int TN>
constexpr size_t m2m_f32_smem() { return MM_NS * (size_t)(MM_TM + TN) * MM_LD * sizeof(float); }
template <int TN>
struct MMShape {
    static constexpr int NT = 10 * TN, PG = TN / 4, NA = MM_TM * (MM_TK / 4) / NT, NB = (TN * MM_TK + NT - 1) / NT;
    static_assert(MM_TM * (MM_TK / 4) % NT == 0, "whole operator copies per thread");
};

// acc[i][j] = sum_{k < K} A[rq + 40 i][k] B[pq + TN/4 j][k] for the operator A (rows < Mrows,
// row stride lda) and the coefficient rows B; bsrc[i] is the row of element e = tid + NT i
// (coefficient row e / 32), already offset by its k = e % 32, or null for a zero row. Returns
// with every copy complete and the block synchronised, so the stages may be reused.
template <int TN, class TI>
__device__ __forceinline__ void mm_term(const float* __restrict__ A, int Mrows, int lda, int K,
                                        const TI* const* bsrc, float* As, float* Bs, float (&acc)[4][4]) {
    using Sh = MMShape<TN>;
    constexpr int NT = Sh::NT, PG = Sh::PG, NA = Sh::NA, NB = Sh::NB;
    const int tid = threadIdx.x, rq = tid / PG, pq = tid % PG;
    const int nit = (K + MM_TK - 1) / MM_TK;   // 1..MM_NS
    // (operator rows past Mrows are never copied: they only feed accumulators that are not used)
#pragma unroll
    for (int it = 0; it < MM_NS; ++it) {   // row e / 8, quad e % 8: a row's 128 bytes per 8 lanes
        if (it < nit) {
#pragma unroll
            for (int i = 0; i < NA; ++i) {
                const int e = tid + NT * i, row = e >> 3, q = e & 7;
                if (row < Mrows) {
                    const uint32_t d = (uint32_t)__cvta_generic_to_shared(As + (it * MM_TM + row) * MM_LD + 4 * q);
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d),
                                 "l"(A + (int64_t)row * lda + it * MM_TK + 4 * q)
                                 : "memory");
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    float rb[MM_NS][NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const TI* src = bsrc[i];
#pragma unroll
        for (int it = 0; it < MM_NS; ++it) {
            const int k = it * MM_TK + ((tid + NT * i) & 31);
            rb[it][i] = (src && k < K) ? (float)src[it * MM_TK] : 0.f;
        }
    }
#pragma unroll
    for (int it = 0; it < MM_NS; ++it)
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int e = tid + NT * i, pp = e >> 5, k = e & 31;
            if (pp < TN) Bs[(it * TN + pp) * MM_LD + k] = rb[it][i];
        }
#pragma unroll
    for (int it = 0; it < MM_NS; ++it) {
        if (it >= nit) break;
        // chunk it's copies are done once at most MM_NS - 1 - it later groups are pending
        if (it == 0) asm volatile("cp.async.wait_group 3;" ::: "memory");
        else if (it == 1) asm volatile("cp.async.wait_group 2;" ::: "memory");
        else if (it == 2) asm volatile("cp.async.wait_group 1;" ::: "memory");
        else asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        const float* Ab = As + (it * MM_TM + rq) * MM_LD;
        const float* Bb = Bs + (it * TN + pq) * MM_LD;
#pragma unroll
        for (int kk = 0; kk < MM_TK; kk += 4) {
            float4 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = *reinterpret_cast<const float4*>(Ab + 40 * i * MM_LD + kk);
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = *reinterpret_cast<const float4*>(Bb + PG * j * MM_LD + kk);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float v = acc[i][j];
                    v = fmaf(a[i].x, b[j].x, v);
                    v = fmaf(a[i].y, b[j].y, v);
                    v = fmaf(a[i].z, b[j].z, v);
                    acc[i][j] = fmaf(a[i].w, b[j].w, v);
                }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();   // every thread is done with the stages
}

// M2M (Eq. (m2m)): chk[parents[p]][s] = sum over the octants o and k < K of
// Mc_o[s][k] c[kids[o][p]][k] (FP32 arithmetic on FP64 coefficients), S <= 160 check points.
// A cluster of 8 blocks takes TN parents, block o of it the octant-o term for every check row
// (mm_term). Each block then leaves its term in its shared memory and, after a cluster
// barrier, sums one eighth of the outputs over the 8 blocks' terms in octant order through
// distributed shared memory: the result does not depend on scheduling.
// (the term's row stride MM_LDP = 4 mod 32: a warp's 8 parents x 4 rows hit 32 banks)
template <int TN>
__global__ void __cluster_dims__(8, 1, 1) __launch_bounds__(10 * TN, 2)
    k_m2m_f32(const float* __restrict__ Mc, int S, int R, int K, const int32_t* __restrict__ kids,
              const int32_t* __restrict__ parents, int count, const double* __restrict__ c, int ldc,
              double* __restrict__ out, int ldo) {
    using Sh = MMShape<TN>;
    constexpr int NT = Sh::NT, PG = Sh::PG, NB = Sh::NB;
    static_assert(TN * MM_LDP <= MM_NS * MM_TM * MM_LD, "the term fits the operator stages");
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) float mm_sm[];
    float* As = mm_sm;                          // [MM_NS][MM_TM][MM_LD]; afterwards the term [TN][MM_LDP]
    float* Bs = mm_sm + MM_NS * MM_TM * MM_LD;  // [MM_NS][TN][MM_LD]
    const int tid = threadIdx.x, o = (int)cl.block_rank(), p0 = (blockIdx.x / 8) * TN;
    const int rq = tid / PG, pq = tid % PG;
    const double* bsrc[NB];   // parent e / 32, k e % 32: a child's row per warp
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int e = tid + NT * i, pp = e >> 5;
        const int ch = (pp < TN && p0 + pp < count) ? kids[(int64_t)o * count + p0 + pp] : -1;
        bsrc[i] = ch >= 0 ? c + (int64_t)ch * ldc + (e & 31) : nullptr;
    }
    float acc[4][4] = {};
    mm_term<TN, double>(Mc + (int64_t)o * S * R, S, R, K, bsrc, As, Bs, acc);
    float* P = As;   // this octant's term, [parent][row]
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) P[(pq + PG * j) * MM_LDP + rq + 40 * i] = acc[i][j];
    cl.sync();
    const float* Pr[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) Pr[r] = cl.map_shared_rank(P, r);
    const int np = min(TN, count - p0);
    for (int e = o * NT + tid; e < np * S; e += 8 * NT) {   // parent e / S, row e % S
        const int pp = e / S, row = e - pp * S;
        float v = 0.f;
#pragma unroll
        for (int r = 0; r < 8; ++r) v += Pr[r][pp * MM_LDP + row];
        out[(int64_t)parents[p0 + pp] * ldo + row] = (double)v;
    }
    cl.sync();   // no block leaves while another reads its term
}

// L2L (Eq. (l2l)) in coefficients, added onto the children's M2L result: for the octant o =
// blockIdx.y, d[dst[zoff[o] + p]][r] += sum_{k < K} Lo_o[r][k] d[src[zoff[o] + p]][k] for
// r < Mo (the child level's rank) and the TN entries p of tile blockIdx.x (mm_term). Each
// output has one term, so no reduction is needed.
template <int TN>
__global__ void __launch_bounds__(10 * TN, 2)
    k_l2l_f32(const float* __restrict__ Lo, int R, int Mo, int K, const int32_t* __restrict__ src,
              const int32_t* __restrict__ dst, const int32_t* __restrict__ zoff, const float* in, float* out) {
    using Sh = MMShape<TN>;
    constexpr int NT = Sh::NT, PG = Sh::PG, NB = Sh::NB;
    extern __shared__ __align__(16) float mm_sm[];
    float* As = mm_sm;
    float* Bs = mm_sm + MM_NS * MM_TM * MM_LD;
    const int o = blockIdx.y, base = zoff[o], count = zoff[o + 1] - base, p0 = blockIdx.x * TN;
    if (p0 >= count) return;   // (the whole block: no barrier is pending)
    const int tid = threadIdx.x, rq = tid / PG, pq = tid % PG;
    const float* bsrc[NB];   // entry e / 32, k e % 32: a parent's row per warp
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int e = tid + NT * i, pp = e >> 5;
        bsrc[i] = (pp < TN && p0 + pp < count) ? in + (int64_t)src[base + p0 + pp] * R + (e & 31) : nullptr;
    }
    float acc[4][4] = {};
    mm_term<TN, float>(Lo + (int64_t)o * R * R, Mo, R, K, bsrc, As, Bs, acc);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int p = p0 + pq + PG * j;
        if (p >= count) continue;
        float* orow = out + (int64_t)dst[base + p] * R;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (rq + 40 * i < Mo) orow[rq + 40 * i] += acc[i][j];
    }
}

template <class F>
static int mm_configure(F* fn, size_t smem, bool& configured) {
    if (!configured) {   // one attribute per instantiation (its size never changes)
        KF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = true;
    }
    return KIFMM_OK;
}

template <int TN>
static int launch_m2m_f32(cudaStream_t st, const float* Mc, int S, int R, int K, const int32_t* kids,
                          const int32_t* parents, int count, const double* c, int ldc, double* out, int ldo) {
    static bool configured = false;
    KF_TRY(mm_configure(k_m2m_f32<TN>, m2m_f32_smem<TN>(), configured));
    k_m2m_f32<TN><<<8u * nbk(count, TN), 10 * TN, m2m_f32_smem<TN>(), st>>>(Mc, S, R, K, kids, parents, count, c,
                                                                           ldc, out, ldo);
    KF_LAUNCH();
    return KIFMM_OK;
}

template <int TN>
static int launch_l2l_f32(cudaStream_t st, const float* Lo, int R, int Mo, int K, const int32_t* src,
                          const int32_t* dst, const int32_t* zoff, int max_count, const float* in, float* out) {
    static bool configured = false;
    KF_TRY(mm_configure(k_l2l_f32<TN>, m2m_f32_smem<TN>(), configured));
    k_l2l_f32<TN><<<dim3(nbk(max_count, TN), 8), 10 * TN, m2m_f32_smem<TN>(), st>>>(Lo, R, Mo, K, src, dst, zoff,
                                                                                   in, out);
    KF_LAUNCH();
    return KIFMM_OK;
}

// tile shapes: FP64 48 x 32 (3 x 2 per thread; ranks near 141 pad to 144), FP32 64 x 64
template <class T> struct ApplyShape;
template <> struct ApplyShape<double> { static constexpr int RM = 3, CN = 2; };
template <> struct ApplyShape<float> { static constexpr int RM = 4, CN = 4; };

// M2L (Eq. (m2l)) in coefficients: d[B] = sum over V(B) of T[slot] c[A], for a tile of
// M2L_TN consecutive boxes of one level, looping over the tile's active offset slots;
// every output belongs to one block. T is [343][R][R] (zero padded), c and d are [nb][R].
// Tile: 64 rows x 64 boxes, k-chunks of 32 (R is a multiple of 32), each thread 4 x 4
// outputs; the next chunk is fetched into registers while the current one is used.
constexpr int M2L_TM = 64, M2L_TN = kM2LTile, M2L_TK = 32;
template <class T>
__global__ void __launch_bounds__(256) k_m2l(const T* __restrict__ Tm, int R, const int32_t* vtab,
                                             const int32_t* slots, int64_t lo, int64_t hi,
                                             const T* __restrict__ c, T* d) {
    __shared__ T As[M2L_TK][M2L_TM + 1];
    __shared__ T Bs[M2L_TK][M2L_TN + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int row0 = blockIdx.y * M2L_TM;
    const int64_t b0 = lo + (int64_t)blockIdx.x * M2L_TN;
    const int32_t* sl = slots + (int64_t)blockIdx.x * kSlotStride;
    const int ns = sl[0];
    const int64_t RR = (int64_t)R * R;
    const int nk = R / M2L_TK;
    const int nsteps = ns * nk;
    // each thread moves 8 elements of A and 8 of B per chunk: element e = tid + 256 i
    T ra[8], rb[8];
    auto fetch = [&](int step) {
        const int si = step / nk, k0 = (step % nk) * M2L_TK;
        const int slot = sl[1 + si];
        const T* Op = Tm + (int64_t)slot * RR;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int e = tid + 256 * i;
            int rr = e / M2L_TK, kk = e % M2L_TK;   // rr < 64: matrix row, and box column for B
            int row = row0 + rr;
            ra[i] = (row < R) ? Op[(int64_t)row * R + k0 + kk] : T(0);
            int64_t b = b0 + rr;
            int a = (b < hi) ? vtab[b * kOffsetSlots + slot] : -1;
            rb[i] = (a >= 0) ? c[(int64_t)a * R + k0 + kk] : T(0);
        }
    };
    T acc[4][4] = {};
    if (nsteps > 0) fetch(0);
    for (int step = 0; step < nsteps; ++step) {
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int e = tid + 256 * i;
            As[e % M2L_TK][e / M2L_TK] = ra[i];
            Bs[e % M2L_TK][e / M2L_TK] = rb[i];
        }
        __syncthreads();
        if (step + 1 < nsteps) fetch(step + 1);
#pragma unroll 8
        for (int kk = 0; kk < M2L_TK; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int row = row0 + ty + 16 * i;
        if (row >= R) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t b = b0 + tx + 16 * j;
            if (b >= hi) continue;
            d[b * R + row] = acc[i][j];
        }
    }
}

__global__ void k_to_f32(const double* in, float* out, int64_t n) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = (float)in[e];
}

// S2L for the X list: downward check potential of B (x_j = c_B + r_in r_B s_j) from the
// sources of every leaf A in X(B). One block per box. Row B of chk (stride ldc) is
// written, or added to when acc != 0 (the Chebyshev representation adds the values at
// B's nodes, x_j = c_B + r_B xbar_j, straight into B's local node values).
template <bool MIXED, class TC>
__global__ void __launch_bounds__(P2M_T) k_s2l_x(EvalView E, const int32_t* boxes, const int32_t* xoff,
                                               const int32_t* xitems, const double* q, TC* chk, int ldc, int acc) {
    const int B = boxes[blockIdx.x];
    const int S = E.S;
    const double r = half_width(E, E.level[B]);
    const double* cB = E.centre + 3 * (int64_t)B;
    __shared__ float4 sp32[256];
    __shared__ double sp64[256][4];
    for (int j0 = 0; j0 < S; j0 += P2M_T) {
        const int j = j0 + threadIdx.x;
        double xj[3];
        for (int k = 0; k < 3; ++k) xj[k] = E.rf_dchk * r * E.surf[3 * min(j, S - 1) + k];
        Kahan acc32;
        double acc64 = 0;
        for (int xi = xoff[B]; xi < xoff[B + 1]; ++xi) {
            const int A = xitems[xi];
            const double* cA = E.centre + 3 * (int64_t)A;
            const float d0 = (float)(cA[0] - cB[0]), d1 = (float)(cA[1] - cB[1]), d2 = (float)(cA[2] - cB[2]);
            for (int s0 = E.pstart[A]; s0 < E.pend[A]; s0 += 256) {
                const int ns = min(256, E.pend[A] - s0);
                __syncthreads();
                for (int e = threadIdx.x; e < ns; e += P2M_T) {
                    if (MIXED) {
                        float4 v = E.loc[s0 + e];
                        sp32[e] = make_float4(v.x + d0, v.y + d1, v.z + d2, (float)q[s0 + e]);
                    } else {
                        for (int k = 0; k < 3; ++k) sp64[e][k] = E.pts[3 * (int64_t)(s0 + e) + k] - cB[k];
                        sp64[e][3] = q[s0 + e];
                    }
                }
                __syncthreads();
                if (MIXED) {
                    const float x0 = (float)xj[0], x1 = (float)xj[1], x2 = (float)xj[2];
                    for (int e = 0; e < ns; ++e) {
                        const float4 v = sp32[e];
                        const float dx = x0 - v.x, dy = x1 - v.y, dz = x2 - v.z;
                        acc32.add(kern_f32(dx * dx + dy * dy + dz * dz, E.kp) * v.w);
                    }
                } else {
                    for (int e = 0; e < ns; ++e) {
                        const double dx = xj[0] - sp64[e][0], dy = xj[1] - sp64[e][1], dz = xj[2] - sp64[e][2];
                        acc64 += kern_f64(sqrt(dx * dx + dy * dy + dz * dz), E.kp) * sp64[e][3];
                    }
                }
            }
        }
        if (j < S) {
            TC* o = chk + (int64_t)B * ldc + j;
            const TC v = (TC)(MIXED ? acc32.value() : acc64);
            *o = acc ? *o + v : v;   // one block per box: no other writer of row B
        }
    }
}

// Targets, far part: local expansion of the leaf (y = c_B + r_out r_B s_k, density phi_d)
// and the W list (y = c_A + r_in r_A s_k, density phi_u). One block per leaf, one thread
// per target point. Writes far[i] for every point of the leaf.
constexpr int L2P_T = 64;
// SER: some target of a leaf may lie closer than 0.5 / (b - a) to its downward equivalent
// surface (the W-list sources always take the series-safe form)
template <bool MIXED, bool SER, class TD>
__global__ void __launch_bounds__(L2P_T) k_l2p(EvalView E, const int32_t* leaves, const int32_t* woff,
                                             const int32_t* witems, const TD* phi_d,
                                             const TD* phi_u, double* far) {
    const int B = leaves[blockIdx.x];
    const int S = E.S;
    const int lev = E.level[B];
    const double* cB = E.centre + 3 * (int64_t)B;
    __shared__ float4 s32[320];
    __shared__ double s64[320][4];
    const int p0 = E.pstart[B], p1 = E.pend[B];
    const int nsrc_lists = 1 + (woff[B + 1] - woff[B]);
    for (int t0 = p0; t0 < p1; t0 += L2P_T) {
        const int i = t0 + threadIdx.x;
        const bool act = i < p1;
        float4 xl = act ? E.loc[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        double x64[3] = {0, 0, 0};
        if (!MIXED && act)
            for (int k = 0; k < 3; ++k) x64[k] = E.pts[3 * (int64_t)i + k] - cB[k];
        Kahan acc32;
        double acc64 = 0;
        for (int li = 0; li < nsrc_lists; ++li) {
            int A;
            double rad;
            const TD* dens;
            int ld = S;
            if (li == 0) {
                if (lev < 2 || E.cheb) continue;   // Chebyshev: interpolation in k_l2p_cheb
                A = B;
                rad = E.rf_out * half_width(E, lev);
                dens = phi_d;
            } else {
                A = witems[woff[B] + li - 1];
                rad = E.rf_ueq * half_width(E, E.level[A]);
                dens = phi_u;
                ld = E.ldu;
            }
            const double* cA = E.centre + 3 * (int64_t)A;
            const double d[3] = {cA[0] - cB[0], cA[1] - cB[1], cA[2] - cB[2]};
            for (int s0 = 0; s0 < S; s0 += 320) {
                const int ns = min(320, S - s0);
                __syncthreads();
                for (int e = threadIdx.x; e < ns; e += L2P_T) {
                    const double* sv = E.surf + 3 * (s0 + e);
                    double y0 = d[0] + rad * sv[0], y1 = d[1] + rad * sv[1], y2 = d[2] + rad * sv[2];
                    double ph = (double)dens[(int64_t)A * ld + s0 + e];
                    if (MIXED) s32[e] = make_float4((float)y0, (float)y1, (float)y2, (float)ph);
                    else {
                        s64[e][0] = y0; s64[e][1] = y1; s64[e][2] = y2; s64[e][3] = ph;
                    }
                }
                __syncthreads();
                if (!act) continue;
                if (MIXED) {
                    const bool plain = !SER && li == 0;
                    int e = 0;
                    for (; e + 7 < ns; e += 8) {   // plain FP32 sums of 8 terms, compensated across blocks
                        float part = 0.f;
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const float4 v = s32[e + u];
                            const float dx = xl.x - v.x, dy = xl.y - v.y, dz = xl.z - v.z;
                            const float r2 = dx * dx + dy * dy + dz * dz;
                            part = fmaf(plain ? kern_plain_f32(r2, E.kp) : kern_f32(r2, E.kp), v.w, part);
                        }
                        acc32.add(part);
                    }
                    for (; e < ns; ++e) {
                        const float4 v = s32[e];
                        const float dx = xl.x - v.x, dy = xl.y - v.y, dz = xl.z - v.z;
                        const float r2 = dx * dx + dy * dy + dz * dz;
                        acc32.add((plain ? kern_plain_f32(r2, E.kp) : kern_f32(r2, E.kp)) * v.w);
                    }
                } else {
                    for (int e = 0; e < ns; ++e) {
                        const double dx = x64[0] - s64[e][0], dy = x64[1] - s64[e][1], dz = x64[2] - s64[e][2];
                        acc64 += kern_f64(sqrt(dx * dx + dy * dy + dz * dz), E.kp) * s64[e][3];
                    }
                }
            }
        }
        if (act) far[i] = MIXED ? acc32.value() : acc64;
    }
}

// ------------------------------------------------------------------------------------
// Chebyshev representation: P2M and the local part of L2P are interpolations
// ------------------------------------------------------------------------------------
// P2M: W_m = sum_j S3(xbar_m, (y_j - c_B) / r_B) q_j for a leaf B, written to out row B
// (stride ldo). One block per leaf; the per-axis weights of a chunk of sources are
// tabulated in shared memory (q_j folded into the x axis), one thread per node m.
constexpr int CP_T = 128, CP_CH = 64;
template <bool MIXED>
__global__ void __launch_bounds__(CP_T) k_p2m_cheb(EvalView E, const int32_t* boxes, const double* q, double* out,
                                                 int ldo) {
    using F = typename std::conditional<MIXED, float, double>::type;
    const int B = boxes[blockIdx.x];
    const int S = E.S, p = E.cp;
    const double r = half_width(E, E.level[B]);
    const int p0 = E.pstart[B], p1 = E.pend[B];
    const double* c = E.centre + 3 * (int64_t)B;
    const F* tab = MIXED ? (const F*)E.ctab32 : (const F*)E.ctab;
    __shared__ F w[3][CP_CH][kChebMaxP];
    for (int j0 = 0; j0 < S; j0 += CP_T) {
        const int j = j0 + threadIdx.x;
        const int jj = min(j, S - 1);
        const int mx = jj % p, my = (jj / p) % p, mz = jj / (p * p);
        Kahan acc32;
        double acc64 = 0;
        for (int s0 = p0; s0 < p1; s0 += CP_CH) {
            const int ns = min(CP_CH, p1 - s0);
            __syncthreads();
            for (int t = threadIdx.x; t < 3 * ns; t += CP_T) {
                const int e = t / 3, a = t % 3;
                F u;
                if (MIXED) {
                    const float4 v = E.loc[s0 + e];
                    u = (F)((a == 0 ? v.x : a == 1 ? v.y : v.z) / (float)r);
                } else {
                    u = (F)((E.pts[3 * (int64_t)(s0 + e) + a] - c[a]) / r);
                }
                F tk[kChebMaxP];
                cheb_T(u, p, tk);
                const F sc = a == 0 ? (F)q[s0 + e] : F(1);
                for (int n = 0; n < p; ++n) w[a][e][n] = sc * cheb_S(tk, p, tab + n * kChebTab);
            }
            __syncthreads();
            if (MIXED) {
                int e = 0;
                for (; e + 7 < ns; e += 8) {   // plain FP32 sums of 8 terms, compensated across blocks
                    float part = 0.f;
#pragma unroll
                    for (int u = 0; u < 8; ++u) part = fmaf((float)(w[0][e + u][mx] * w[1][e + u][my]), (float)w[2][e + u][mz], part);
                    acc32.add(part);
                }
                for (; e < ns; ++e) acc32.add((float)(w[0][e][mx] * w[1][e][my] * w[2][e][mz]));
            } else {
                for (int e = 0; e < ns; ++e) acc64 += (double)w[0][e][mx] * (double)w[1][e][my] * (double)w[2][e][mz];
            }
        }
        if (j < S) out[(int64_t)B * ldo + j] = MIXED ? acc32.value() : acc64;
    }
}

// L2P, local part: far[i] += sum_m S3(xbar_m, (x_i - c_B) / r_B) g^B_m for every point of a
// leaf B at level >= 2 (g row B of stride ldg), summed axis by axis (x innermost). One
// block per leaf, one thread per target; the node values of B and each thread's per-axis
// weights sit in shared memory.
template <bool MIXED, class TD>
__global__ void __launch_bounds__(L2P_T) k_l2p_cheb(EvalView E, const int32_t* leaves, const TD* g, int ldg,
                                                  double* far) {
    using F = typename std::conditional<MIXED, float, double>::type;
    const int B = leaves[blockIdx.x];
    const int lev = E.level[B];
    if (lev < 2) return;
    const int S = E.S, p = E.cp;
    const double r = half_width(E, lev);
    const double* cB = E.centre + 3 * (int64_t)B;
    const F* tab = MIXED ? (const F*)E.ctab32 : (const F*)E.ctab;
    __shared__ F gs[kChebMaxP * kChebMaxP * kChebMaxP];
    __shared__ F sw[3][kChebMaxP][L2P_T];
    for (int m = threadIdx.x; m < S; m += L2P_T) gs[m] = (F)g[(int64_t)B * ldg + m];
    __syncthreads();
    const int p0 = E.pstart[B], p1 = E.pend[B];
    const int tx = threadIdx.x;
    for (int i = p0 + tx; i < p1; i += L2P_T) {
        for (int a = 0; a < 3; ++a) {
            F u;
            if (MIXED) {
                const float4 v = E.loc[i];
                u = (F)((a == 0 ? v.x : a == 1 ? v.y : v.z) / (float)r);
            } else {
                u = (F)((E.pts[3 * (int64_t)i + a] - cB[a]) / r);
            }
            F tk[kChebMaxP];
            cheb_T(u, p, tk);
            for (int n = 0; n < p; ++n) sw[a][n][tx] = cheb_S(tk, p, tab + n * kChebTab);
        }
        F acc = 0;
        for (int mz = 0; mz < p; ++mz) {
            F accy = 0;
            for (int my = 0; my < p; ++my) {
                const F* row = gs + (mz * p + my) * p;
                F accx = 0;
                for (int mx = 0; mx < p; ++mx) accx += sw[0][mx][tx] * row[mx];
                accy += sw[1][my][tx] * accx;
            }
            acc += sw[2][mz][tx] * accy;
        }
        far[i] += (double)acc;
    }
}

// Chebyshev M2M and L2L by the tensor-product structure of the interpolation:
//   M_o = A[oz] (x) A[oy] (x) A[ox],  A[b][n][m] = S(0.5 (2b - 1) + 0.5 xbar_m, xbar_n),
// applied as three passes of p-term sums (x, then y, then z): 3 p^4 instead of p^6 products.
constexpr int KR_T = 256, KR_MAXS = kChebMaxP * kChebMaxP * kChebMaxP;
// W^P = sum_o M_o W^{C_o} for the listed parents (node weights in cu, rows of stride R);
// one block per parent, arithmetic in F
template <class F>
__global__ void __launch_bounds__(KR_T) k_cheb_m2m_kron(const int32_t* __restrict__ parents,
                                                      const int32_t* __restrict__ child, const double* __restrict__ Ag,
                                                      int p, double* cu, int R) {
    const int P = parents[blockIdx.x];
    const int S = p * p * p, p2 = p * p;
    __shared__ F A[2 * kChebMaxP * kChebMaxP];
    __shared__ F w[KR_MAXS], t1[KR_MAXS], t2[KR_MAXS];
    for (int e = threadIdx.x; e < 2 * p2; e += KR_T) A[e] = (F)Ag[e];
    F acc[(KR_MAXS + KR_T - 1) / KR_T] = {};
    for (int o = 0; o < 8; ++o) {
        const int C = child[8 * (int64_t)P + o];
        if (C < 0) continue;   // the same for the whole block
        const F* Ax = A + (o & 1) * p2;
        const F* Ay = A + ((o >> 1) & 1) * p2;
        const F* Az = A + ((o >> 2) & 1) * p2;
        __syncthreads();
        for (int n = threadIdx.x; n < S; n += KR_T) w[n] = (F)cu[(int64_t)C * R + n];
        __syncthreads();
        for (int n = threadIdx.x; n < S; n += KR_T) {   // t1[mz][my][nx] = sum_mx A_x[nx][mx] w[mz][my][mx]
            const int nx = n % p, r = n - nx;
            F v = 0;
            for (int m = 0; m < p; ++m) v += Ax[nx * p + m] * w[r + m];
            t1[n] = v;
        }
        __syncthreads();
        for (int n = threadIdx.x; n < S; n += KR_T) {   // t2[mz][ny][nx] = sum_my A_y[ny][my] t1[mz][my][nx]
            const int nx = n % p, ny = (n / p) % p, mz = n / p2;
            F v = 0;
            for (int m = 0; m < p; ++m) v += Ay[ny * p + m] * t1[mz * p2 + m * p + nx];
            t2[n] = v;
        }
        __syncthreads();
        for (int k = 0, n = threadIdx.x; n < S; ++k, n += KR_T) {   // += sum_mz A_z[nz][mz] t2[mz][ny][nx]
            const int nz = n / p2, q = n % p2;
            F v = 0;
            for (int m = 0; m < p; ++m) v += Az[nz * p + m] * t2[m * p2 + q];
            acc[k] += v;
        }
    }
    for (int k = 0, n = threadIdx.x; n < S; ++k, n += KR_T) cu[(int64_t)P * R + n] = (double)acc[k];
}

// g^C += M_o^T g^P for the boxes lo .. lo + gridDim.x - 1 (all of one level >= 3; o the box's
// octant in its parent), local node values in d (rows of stride R); one block per box
template <class TD>
__global__ void __launch_bounds__(KR_T) k_cheb_l2l_kron(int64_t lo, const int32_t* __restrict__ parent,
                                                      const int32_t* __restrict__ anchor, const double* __restrict__ Ag,
                                                      int p, TD* d, int R) {
    using F = TD;
    const int64_t C = lo + blockIdx.x;
    const int P = parent[C];
    const int o = (anchor[3 * C] & 1) | ((anchor[3 * C + 1] & 1) << 1) | ((anchor[3 * C + 2] & 1) << 2);
    const int S = p * p * p, p2 = p * p;
    __shared__ F A[2 * kChebMaxP * kChebMaxP];
    __shared__ F g[KR_MAXS], t1[KR_MAXS], t2[KR_MAXS];
    for (int e = threadIdx.x; e < 2 * p2; e += KR_T) A[e] = (F)Ag[e];
    for (int n = threadIdx.x; n < S; n += KR_T) g[n] = d[(int64_t)P * R + n];
    __syncthreads();
    const F* Ax = A + (o & 1) * p2;
    const F* Ay = A + ((o >> 1) & 1) * p2;
    const F* Az = A + ((o >> 2) & 1) * p2;
    for (int m = threadIdx.x; m < S; m += KR_T) {   // t1[nz][ny][mx] = sum_nx A_x[nx][mx] g[nz][ny][nx]
        const int mx = m % p, r = m - mx;
        F v = 0;
        for (int n = 0; n < p; ++n) v += Ax[n * p + mx] * g[r + n];
        t1[m] = v;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < S; m += KR_T) {   // t2[nz][my][mx] = sum_ny A_y[ny][my] t1[nz][ny][mx]
        const int mx = m % p, my = (m / p) % p, nz = m / p2;
        F v = 0;
        for (int n = 0; n < p; ++n) v += Ay[n * p + my] * t1[nz * p2 + n * p + mx];
        t2[m] = v;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < S; m += KR_T) {   // d^C[mz][my][mx] += sum_nz A_z[nz][mz] t2[nz][my][mx]
        const int mz = m / p2, q = m % p2;
        F v = 0;
        for (int n = 0; n < p; ++n) v += Az[n * p + mz] * t2[n * p2 + q];
        d[C * R + m] += v;
    }
}

// Near field (Eq. (nearfar), first sum) over U(B), plus the far part, the self term and
// the scale C; writes the result in the caller's order. One block per leaf:
// 64 targets x 4 source groups; sources staged in shared memory, B-local coordinates.
constexpr int P2P_T = 256, P2P_TGT = 64, P2P_GRP = P2P_T / P2P_TGT, P2P_CHUNK = 2048;
template <bool MIXED, class TO>
__global__ void __launch_bounds__(P2P_T) k_p2p(EvalView E, const int32_t* leaves, const int32_t* uoff,
                                             const int32_t* uitems, const double* q, const double* far,
                                             const double* sigma, const double* Is, const int32_t* perm,
                                             double C, TO* out) {
    const int B = leaves[blockIdx.x];
    const double* cB = E.centre + 3 * (int64_t)B;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* s32 = reinterpret_cast<float4*>(smem_raw);
    double* s64 = reinterpret_cast<double*>(smem_raw);
    __shared__ double red[P2P_GRP][P2P_TGT];
    const int p0 = E.pstart[B], p1 = E.pend[B];
    const int tl = threadIdx.x % P2P_TGT, g = threadIdx.x / P2P_TGT;
    const int u0 = uoff[B], u1 = uoff[B + 1];
    const int chunk = MIXED ? P2P_CHUNK : P2P_CHUNK / 2;
    for (int t0 = p0; t0 < p1; t0 += P2P_TGT) {
        const int i = t0 + tl;
        const bool act = i < p1;
        float4 xl = act ? E.loc[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        double x64[3] = {0, 0, 0};
        if (!MIXED && act)
            for (int k = 0; k < 3; ++k) x64[k] = E.pts[3 * (int64_t)i + k] - cB[k];
        Kahan acc32;
        double acc64 = 0;
        // walk the U list in chunks of sources
        int ui = u0, uoffs = 0;
        while (ui < u1) {
            __syncthreads();
            int ns = 0;
            // stage: every thread walks the same boxes, writing its share
            int wi = ui, wo = uoffs;
            while (wi < u1 && ns < chunk) {
                const int A = uitems[wi];
                const int a0 = E.pstart[A], a1 = E.pend[A];
                const int take = min(a1 - a0 - wo, chunk - ns);
                const double* cA = E.centre + 3 * (int64_t)A;
                if (MIXED) {
                    const float d0 = (float)(cA[0] - cB[0]), d1 = (float)(cA[1] - cB[1]), d2 = (float)(cA[2] - cB[2]);
                    for (int e = threadIdx.x; e < take; e += P2P_T) {
                        float4 v = E.loc[a0 + wo + e];
                        s32[ns + e] = make_float4(v.x + d0, v.y + d1, v.z + d2, (float)q[a0 + wo + e]);
                    }
                } else {
                    for (int e = threadIdx.x; e < take; e += P2P_T) {
                        int64_t j = a0 + wo + e;
                        s64[4 * (ns + e) + 0] = E.pts[3 * j] - cB[0];
                        s64[4 * (ns + e) + 1] = E.pts[3 * j + 1] - cB[1];
                        s64[4 * (ns + e) + 2] = E.pts[3 * j + 2] - cB[2];
                        s64[4 * (ns + e) + 3] = q[j];
                    }
                }
                ns += take;
                wo += take;
                if (wo >= a1 - a0) {
                    ++wi;
                    wo = 0;
                }
            }
            __syncthreads();
            if (act) {
                if (MIXED) {
                    for (int e = g; e < ns; e += P2P_GRP) {
                        const float4 v = s32[e];
                        const float dx = xl.x - v.x, dy = xl.y - v.y, dz = xl.z - v.z;
                        const float r2 = dx * dx + dy * dy + dz * dz;
                        // j == i gives r2 == 0 exactly (same FP32 arithmetic); points are distinct
                        if (r2 > 0.f) acc32.add(kern_f32(r2, E.kp) * v.w);
                    }
                } else {
                    for (int e = g; e < ns; e += P2P_GRP) {
                        const double dx = x64[0] - s64[4 * e], dy = x64[1] - s64[4 * e + 1],
                                     dz = x64[2] - s64[4 * e + 2];
                        const double r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 > 0.0) acc64 += kern_f64(sqrt(r2), E.kp) * s64[4 * e + 3];
                    }
                }
            }
            ui = wi;
            uoffs = wo;
        }
        red[g][tl] = MIXED ? acc32.value() : acc64;
        __syncthreads();
        if (g == 0 && act) {
            double s = 0;
            for (int k = 0; k < P2P_GRP; ++k) s += red[k][tl];
            double v = C * (s + far[i] + sigma[i] * Is[i]);
            if (perm[i] < E.n_real) out[perm[i]] = (TO)v;
        }
        __syncthreads();
    }
}

// Near field, mixed form: the same sum as k_p2p<true> with two targets per thread, so that
// every source read from shared memory serves two pair evaluations. 128 threads per leaf:
// lane = target pair (targets t and t + 32 of a 64-target chunk), warp = source group.
// Sources carry q * norm, so a pair costs (e^{-aR} - e^{-bR}) * (q norm) / R^3.
// SERIES: some pair of the plan is closer than 0.5 / (b - a), where the factored form with
// the series of 1 - e^{-(b-a)R} is needed; otherwise every pair takes the plain difference
// of the two exponentials. GUARD: the sources are the target's own box, which holds the
// target itself (r2 == 0 exactly: points are distinct), whose term is dropped.
constexpr int P2Q_T = 128, P2Q_GRP = 4, P2Q_CHUNK = 1024;   // 16 KB of sources per block
constexpr int P2Q_BLK = 8;   // plain FP32 partial sums of 8 pairs, compensated across partial sums
template <bool SERIES, bool GUARD>
__device__ __forceinline__ float p2q_term(const float4& x, const float4& v, const KParams& kp, float acc) {
    const float dx = x.x - v.x, dy = x.y - v.y, dz = x.z - v.z;
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float rinv = rsqrt_approx(r2);
    const float R = r2 * rinv;
    const float w = v.w * rinv * (rinv * rinv);
    float ed;
    if (SERIES) ed = exp_diff_f32(R, kp);
    else ed = ex2_approx(-kp.a_l2e * R) - ex2_approx(-kp.b_l2e * R);
    if (GUARD) return r2 > 0.f ? fmaf(ed, w, acc) : acc;
    return fmaf(ed, w, acc);
}

template <bool SERIES, class TO>
__global__ void __launch_bounds__(P2Q_T) k_p2p_mixed(EvalView E, const int32_t* leaves, const int32_t* uoff,
                                                     const int32_t* uitems, const double* q, const double* far,
                                                     const double* sigma, const double* Is, const int32_t* perm,
                                                     double C, TO* out) {
    const int B = leaves[blockIdx.x];
    const double* cB = E.centre + 3 * (int64_t)B;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* s32 = reinterpret_cast<float4*>(smem_raw);
    __shared__ double red[P2Q_GRP][64];
    const int p0 = E.pstart[B], p1 = E.pend[B];
    const int tp = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int u0 = uoff[B], u1 = uoff[B + 1];
    const float nrm = E.kp.norm_f;
    for (int t0 = p0; t0 < p1; t0 += 64) {
        const int i0 = t0 + tp, i1 = t0 + tp + 32;
        const bool a0 = i0 < p1, a1 = i1 < p1;
        const float4 far4 = make_float4(1e30f, 1e30f, 1e30f, 0.f);   // inactive slot: never near a source
        const float4 x0 = a0 ? E.loc[i0] : far4, x1 = a1 ? E.loc[i1] : far4;
        Kahan k0, k1;
        // the source boxes in the order: B itself (index u0 - 1), then U(B) without B
        int ui = u0 - 1, uoffs = 0, own_left = p1 - p0;
        while (ui < u1) {
            __syncthreads();
            int ns = 0, wi = ui, wo = uoffs;
            while (wi < u1 && ns < P2Q_CHUNK) {
                const int A = wi < u0 ? B : uitems[wi];
                if (wi >= u0 && A == B) {
                    ++wi;
                    continue;
                }
                const int aa = E.pstart[A], ab = E.pend[A];
                const int take = min(ab - aa - wo, P2Q_CHUNK - ns);
                const double* cA = E.centre + 3 * (int64_t)A;
                const float d0 = (float)(cA[0] - cB[0]), d1 = (float)(cA[1] - cB[1]), d2 = (float)(cA[2] - cB[2]);
                for (int e = threadIdx.x; e < take; e += P2Q_T) {
                    const float4 v = E.loc[aa + wo + e];
                    s32[ns + e] = make_float4(v.x + d0, v.y + d1, v.z + d2, (float)q[aa + wo + e] * nrm);
                }
                ns += take;
                wo += take;
                if (wo >= ab - aa) {
                    ++wi;
                    wo = 0;
                }
            }
            __syncthreads();
            const int n_own = min(own_left, ns);   // the chunk's leading sources are B's own points
            own_left -= n_own;
            int e = g;
            for (; e < n_own; e += P2Q_GRP) {
                const float4 v = s32[e];
                k0.add(p2q_term<SERIES, true>(x0, v, E.kp, 0.f));
                k1.add(p2q_term<SERIES, true>(x1, v, E.kp, 0.f));
            }
            for (; e + (P2Q_BLK - 1) * P2Q_GRP < ns; e += P2Q_BLK * P2Q_GRP) {
                float s0 = 0.f, s1 = 0.f;
#pragma unroll
                for (int u = 0; u < P2Q_BLK; ++u) {
                    const float4 v = s32[e + u * P2Q_GRP];
                    s0 = p2q_term<SERIES, false>(x0, v, E.kp, s0);
                    s1 = p2q_term<SERIES, false>(x1, v, E.kp, s1);
                }
                k0.add(s0);
                k1.add(s1);
            }
            {
                float s0 = 0.f, s1 = 0.f;
                for (; e < ns; e += P2Q_GRP) {
                    const float4 v = s32[e];
                    s0 = p2q_term<SERIES, false>(x0, v, E.kp, s0);
                    s1 = p2q_term<SERIES, false>(x1, v, E.kp, s1);
                }
                k0.add(s0);
                k1.add(s1);
            }
            ui = wi;
            uoffs = wo;
        }
        red[g][tp] = k0.value();
        red[g][tp + 32] = k1.value();
        __syncthreads();
        if (g < 2) {
            const int tl = tp + 32 * g;
            const int i = t0 + tl;
            if (i < p1) {
                double s = 0;
                for (int k = 0; k < P2Q_GRP; ++k) s += red[k][tl];
                if (perm[i] < E.n_real) out[perm[i]] = (TO)(C * (s + far[i] + sigma[i] * Is[i]));
            }
        }
        __syncthreads();
    }
}

// Plan time: the smallest squared distance (box-local FP32 coordinates, as in the pair
// kernel) between two distinct points of one U pair, as float bits into *minbits.
__global__ void __launch_bounds__(128) k_min_r2(EvalView E, const int32_t* leaves, const int32_t* uoff,
                                                const int32_t* uitems, unsigned int* minbits) {
    const int B = leaves[blockIdx.x];
    const double* cB = E.centre + 3 * (int64_t)B;
    const int p0 = E.pstart[B], p1 = E.pend[B];
    float m = 3.0e38f;
    for (int k = uoff[B]; k < uoff[B + 1]; ++k) {
        const int A = uitems[k];
        const double* cA = E.centre + 3 * (int64_t)A;
        const float d0 = (float)(cA[0] - cB[0]), d1 = (float)(cA[1] - cB[1]), d2 = (float)(cA[2] - cB[2]);
        const int aa = E.pstart[A], ab = E.pend[A];
        for (int i = p0 + (int)threadIdx.x; i < p1; i += blockDim.x) {
            const float4 x = E.loc[i];
            for (int j = aa; j < ab; ++j) {
                if (j == i) continue;
                const float4 v = E.loc[j];
                const float dx = x.x - (v.x + d0), dy = x.y - (v.y + d1), dz = x.z - (v.z + d2);
                m = fminf(m, dx * dx + dy * dy + dz * dz);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMin(minbits, __float_as_uint(m));
}

// ------------------------------------------------------------------------------------
// driver
// ------------------------------------------------------------------------------------
static EvalView make_view(Plan& p) {
    EvalView E;
    E.pts = ptr<double>(p.pts);
    E.loc = ptr<float4>(p.loc32);
    E.centre = ptr<double>(p.tree.centre);
    E.level = ptr<int32_t>(p.tree.level);
    E.pstart = ptr<int32_t>(p.tree.pstart);
    E.pend = ptr<int32_t>(p.tree.pend);
    E.surf = ptr<double>(p.surf);
    E.side = p.tree.side;
    E.S = p.S;
    E.kp = make_kparams_kind(p.kind, p.a, p.b);
    E.cheb = p.cheb ? 1 : 0;
    E.rf_dchk = p.cheb ? 1.0 : p.r_in;
    E.rf_ueq = p.cheb ? 1.0 : p.r_in;
    E.rf_out = p.r_out;
    E.ldu = p.cheb ? p.R : p.S;
    E.cp = p.m0;
    E.ctab = ptr<double>(p.ctab);
    E.ctab32 = ptr<float>(p.ctab32);
    E.n_real = p.n_real;
    return E;
}

// Whether any near pair is closer than 0.5 / (b - a) (with a 1 % margin), where the mixed
// pair kernel needs the series form of 1 - e^{-(b-a)R}.
static int p2p_series_check(Plan& p) {
    p.p2p_series = true;
    if (p.nleaves <= 0) return KIFMM_OK;
    DevBuf mb;
    KF_TRY(dev_alloc(mb, 4));
    const unsigned int init = 0x7f7fffffu;   // largest finite float
    KF_CUDA(cudaMemcpyAsync(mb.p, &init, 4, cudaMemcpyHostToDevice, p.stream));
    EvalView E = make_view(p);
    k_min_r2<<<(unsigned)p.nleaves, 128, 0, p.stream>>>(E, ptr<int32_t>(p.leaves), ptr<int32_t>(p.lists[0].off),
                                                        ptr<int32_t>(p.lists[0].items), ptr<unsigned int>(mb));
    KF_LAUNCH();
    unsigned int bits = 0;
    KF_CUDA(cudaMemcpyAsync(&bits, mb.p, 4, cudaMemcpyDeviceToHost, p.stream));
    KF_CUDA(cudaStreamSynchronize(p.stream));
    dev_free(mb);
    float m;
    std::memcpy(&m, &bits, 4);
    const double rs = 1.01 * 0.5 / (p.b - p.a);
    p.p2p_series = !((double)m >= rs * rs);
    // leaves' points lie within their box (half-width r), their check / equivalent surfaces
    // at r_out r: every such pair is at least (r_out - 1) r apart
    double rmin = 1e300;
    for (int l = 2; l < p.tree.nlevels; ++l)
        if (p.lv[l].n_leaf > 0) rmin = std::min(rmin, p.tree.side / (double)(2LL << l));
    p.far_series = !((p.r_out - 1.0) * rmin >= rs);
    return KIFMM_OK;
}

// Phase boundaries of one evaluation: k = 0..7 opens phase k (scatter, S2M, M2M + UC2UE, M2L,
// S2L + L2L + DC2DE, L2P + M2P, P2P) and closes the open one. A CUDA event per boundary when
// the plan times its phases, and a named NVTX range per phase on the host (no-ops unless a
// profiler is attached; a range left open by a failed evaluation closes at the next mark).
static const char* const kPhaseNames[7] = {"kifmm scatter", "kifmm S2M", "kifmm M2M+UC2UE", "kifmm M2L",
                                           "kifmm S2L+L2L+DC2DE", "kifmm L2P+M2P", "kifmm P2P"};
static void mark(Plan& p, int k) {
    if (p.timing) cudaEventRecord(p.ev[k], p.stream);
    if (p.nvtx_range) {
        nvtxRangeEnd(p.nvtx_range);
        p.nvtx_range = 0;
    }
    if (k < 7) p.nvtx_range = nvtxRangeStartA(kPhaseNames[k]);
}

template <class T> static const T* sel(const DevBuf& d64, const DevBuf& d32);
template <> const double* sel<double>(const DevBuf& d64, const DevBuf&) { return ptr<double>(d64); }
template <> const float* sel<float>(const DevBuf&, const DevBuf& d32) { return ptr<float>(d32); }

// Op has row stride ldop; only its leading Mo x Ki block is applied (the rest is zero padding).
// nz > 1 without zoff splits the terms over nz slices that add atomically into out.
template <class T, class TI = T, class TO = T>
static int launch_apply(cudaStream_t st, const T* Op, int ldop, int Mo, int Ki, const int32_t* src, const int32_t* dst,
                        int64_t base, int count, const TI* in, int ldi, TO* out, int ldo, int acc, int nterm = 1,
                        int64_t op_stride = 0, const int32_t* zoff = nullptr, int nz = 1, int64_t zstride = 0,
                        DevBuf* part = nullptr, int64_t* nl = nullptr) {
    if (count <= 0) return KIFMM_OK;
    constexpr int RM = ApplyShape<T>::RM, CN = ApplyShape<T>::CN;
    dim3 g(nbk(count, 16 * CN), nbk(Mo, 16 * RM), nz);
    const int64_t ncp = (int64_t)g.x * 16 * CN, nrp = (int64_t)g.y * 16 * RM;
    TO* pp = nullptr;
    // the split's partial sums, added in order by k_apply_finish (the work space is sized at plan
    // time for a split of at most one wave; nothing is allocated here, so evaluations can be
    // captured in a graph)
    if (nz > 1 && !zoff && part && part->bytes >= (size_t)nz * ncp * nrp * sizeof(TO)) pp = static_cast<TO*>(part->p);
    k_apply<T, TI, TO, RM, CN><<<g, 256, 0, st>>>(Op, op_stride, ldop, nterm, Mo, Ki, src, dst, base, count, in, ldi,
                                                  out, ldo, acc, zoff, zstride, pp);
    KF_LAUNCH();
    if (pp) {
        k_apply_finish<TO><<<nbk((int64_t)count * Mo, 256), 256, 0, st>>>(pp, nz, ncp, (int)nrp, count, Mo, dst, base,
                                                                         out, ldo, acc);
        KF_LAUNCH();
        if (nl) ++*nl;
    }
    return KIFMM_OK;
}

// Far field: upward pass (FP64 in both forms), M2L, downward pass and the leaves'
// downward equivalent densities, in type T (FP64 form: double; mixed form: float).
// the near sums on the plan's second stream, after the work ordered before near_ev[0] on the
// plan's stream; near_ev[1] is recorded whatever happened, so that a join never waits on an
// unrecorded event and a capture never holds an open fork
static int near_fork_launch(Plan& p, int64_t& nl) {
    cudaError_t e = cudaStreamWaitEvent(p.near_st, p.near_ev[0], 0);
    int rc = KIFMM_OK;
    if (e != cudaSuccess) {
        set_error(std::string("near-field fork: ") + cudaGetErrorString(e));
        return KIFMM_ERR_CUDA;
    }
    p.near_forked = true;
    p.near_pending = false;
    if (p.timing && p.near_tev[0]) cudaEventRecord(p.near_tev[0], p.near_st);
    rc = near_tc_contract(p, p.near_st, nl);
    if (p.timing && p.near_tev[1]) cudaEventRecord(p.near_tev[1], p.near_st);
    e = cudaEventRecord(p.near_ev[1], p.near_st);
    if (rc == KIFMM_OK && e != cudaSuccess) {
        set_error(std::string("near-field fork: ") + cudaGetErrorString(e));
        rc = KIFMM_ERR_CUDA;
    }
    return rc;
}

template <class T>
static int run_far(Plan& p, const EvalView& E, int64_t& nl) {
    Tree& t = p.tree;
    cudaStream_t st = p.stream;
    const int S = p.S, R = p.R, L = t.nlevels;
    const bool mixed = p.precision == KIFMM_MIXED;
    double* cu = ptr<double>(p.cu);
    T* dd = ptr<T>(p.dd);
    T* phid = ptr<T>(p.phid);
#define RUN(x)     \
    do {           \
        KF_TRY(x); \
        ++nl;      \
    } while (0)
    // ---- upward (Eqs. (s2m), (m2m)): check potentials of the leaves from their sources (S2M)
    // and of the parents from their children's coefficients (M2M to the parent's upward check
    // surface, in T), then c = Sigma^+ U^T chk for every box (the pseudo-inverse, FP64), level
    // by level from the deepest
    KF_CUDA(cudaMemsetAsync(cu, 0, (size_t)t.nboxes * R * 8, st));
    if (L - 1 > 2) {   // parents' check rows, accumulated atomically where the terms are split
        const int64_t b0 = t.level_start[2], b1 = t.level_start[L - 1];
        KF_CUDA(cudaMemsetAsync(ptr<double>(p.chk) + b0 * S, 0, (size_t)(b1 - b0) * S * 8, st));
    }
    if (p.n_p2m > 0 && p.cheb && p.lat_far) {   // lattice: one interpolation matrix for every leaf
        KF_TRY(lat_s2m(p));
        ++nl;
    } else if (p.n_p2m > 0 && p.cheb) {   // node weights of the leaves, straight into c
        auto* kp2m = mixed ? k_p2m_cheb<true> : k_p2m_cheb<false>;
        kp2m<<<(unsigned)p.n_p2m, CP_T, 0, st>>>(E, ptr<int32_t>(p.p2m_boxes), ptr<double>(p.q), cu, R);
        KF_LAUNCH();
        ++nl;
    } else if (p.n_p2m > 0 && p.lat_far) {   // uniform lattice: one check matrix for every leaf
        if (!p.lat_up) {                      // (else the leaves' c come straight from q below)
            KF_TRY(lat_s2m(p));
            ++nl;
        }
    } else if (p.n_p2m > 0) {
        auto* kp2m = !mixed ? k_p2m<false, true> : (p.far_series ? k_p2m<true, true> : k_p2m<true, false>);
        kp2m<<<(unsigned)p.n_p2m, P2M_T, 0, st>>>(E, ptr<int32_t>(p.p2m_boxes), ptr<double>(p.q), ptr<double>(p.chk));
        KF_LAUNCH();
        ++nl;
    }
    mark(p, 2);
    for (int l = L - 1; l >= 2; --l) {
        auto& LL = p.lv[l];
        if (LL.n_par > 0 && p.cheb) {   // Chebyshev: three 1-D passes per child, straight into c
            if (mixed)
                k_cheb_m2m_kron<float><<<LL.n_par, KR_T, 0, st>>>(ptr<int32_t>(LL.parents), ptr<int32_t>(t.child),
                                                                  ptr<double>(p.cheb_A), p.m0, cu, R);
            else
                k_cheb_m2m_kron<double><<<LL.n_par, KR_T, 0, st>>>(ptr<int32_t>(LL.parents), ptr<int32_t>(t.child),
                                                                   ptr<double>(p.cheb_A), p.m0, cu, R);
            KF_LAUNCH();
            ++nl;
        } else if (LL.n_par > 0 && mixed && p.m2m_tc && p.m2m_count[l] >= p.tc_min_tiles) {
            // tensor cores: the children's c split FP16 x 3 (the M2L operand buffers, rewritten
            // before M2L), 8 octant slots per parent tile, staged in FP32, copied to the check rows
            const int64_t lo = t.level_start[l + 1], cnt = t.level_start[l + 2] - lo;
            const int Mt = p.m2m_R;
            void* hi = Mt > R ? p.m2m_hi.p : p.chi.p;
            void* lo16 = Mt > R ? p.m2m_lo.p : p.clo.p;
            KF_TRY(m2l_tc_split_pad(st, cu + lo * R, cnt, R, Mt, static_cast<char*>(hi) + lo * Mt * 2,
                                    static_cast<char*>(lo16) + lo * Mt * 2, ptr<int>(p.cexp) + lo));
            ++nl;
            M2LTables tabs{};
            tabs.hi[l] = p.ops[l].Mhi.p;
            tabs.lo[l] = p.ops[l].Mlo.p;
            tabs.sT[l] = p.ops[l].m2m_sT;
            RUN(launch_tc_translate(st, tabs, Mt, ptr<int4>(p.m2m_tiles) + p.m2m_first[l], p.m2m_count[l],
                                    ptr<int32_t>(LL.parents), ptr<int32_t>(t.child), 8,
                                    ptr<int32_t>(p.m2m_slots) + (int64_t)p.m2m_first[l] * kSlotStride, hi, lo16,
                                    ptr<int>(p.cexp), ptr<float>(p.stage32), 0, ptr<int>(p.err)));
            rows_f2d<<<nbk((int64_t)LL.n_par * S, 256), 256, 0, st>>>(ptr<int32_t>(LL.parents), LL.n_par,
                                                                     ptr<float>(p.stage32), Mt,
                                                                     p.cheb ? cu : ptr<double>(p.chk),
                                                                     p.cheb ? R : S, S);
            KF_LAUNCH();
            ++nl;
        } else if (LL.n_par > 0 && mixed && S <= MM_TM && p.ops[l + 1].rank <= MM_NS * MM_TK) {
            // chk[P] = sum_o Mc_{l,o} c[C_o], FP32
            // (32 parents a cluster where that gives every SM two blocks, else 16)
            auto* fn = 8 * nbk(LL.n_par, 32) >= 2u * p.num_sms ? launch_m2m_f32<32> : launch_m2m_f32<16>;
            KF_TRY(fn(st, ptr<float>(p.ops[l].Mc32), S, R, p.ops[l + 1].rank, ptr<int32_t>(LL.par_kids),
                      ptr<int32_t>(LL.parents), LL.n_par, cu, R, ptr<double>(p.chk), S));
            ++nl;
        } else if (LL.n_par > 0) {   // chk[P] = sum_o Mc_{l,o} c[C_o]; the 8 octant terms split over z on small levels
            constexpr int RMt = ApplyShape<T>::RM, CNt = ApplyShape<T>::CN;
            const int tiles = (int)(nbk(LL.n_par, 16 * CNt) * nbk(S, 16 * RMt));
            // split the terms so that the launch is one whole wave (4 blocks of 256 per SM at 64
            // registers): a partial second wave costs a wave of latency
            const int nz = std::max(1, std::min(16, std::min(8 * (int)nbk(p.ops[l + 1].rank, AP_TK), (4 * p.num_sms) / tiles)));
            // (Chebyshev: the parents' node weights W^P = sum_o M_o W^{C_o}, straight into c)
            RUN((launch_apply<T, double, double>(st, sel<T>(p.ops[l].Mc, p.ops[l].Mc32), R, S, p.ops[l + 1].rank,
                                                 ptr<int32_t>(LL.par_kids), ptr<int32_t>(LL.parents), 0, LL.n_par,
                                                 cu, R, p.cheb ? cu : ptr<double>(p.chk), p.cheb ? R : S, 0, 8,
                                                 (int64_t)S * R, nullptr, nz, 0, &p.apply_part, &nl)));
        }
        if (p.cheb) continue;   // no pseudo-inverse
        if (p.lat_up && l == p.nf_level) {   // lattice leaves: c = (G1 P) q, FP64-exact on the tensor cores
            KF_TRY(lat_up_apply(p, cu, nl));
        } else if (LL.n_up > p.oz_min && p.oz) {   // c = Sigma^+ U^T chk, FP64-exact on the tensor cores
            int64_t extra = 0;
            KF_TRY(pinv_oz_apply(st, ptr<double>(p.chk), S, ptr<int32_t>(LL.upb), nullptr, LL.n_up, p.ops[l].ozG1.p,
                                 ptr<int>(p.ops[l].ozEr), p.ops[l].rank, p.ozBox.p, ptr<int>(p.ozEb), cu, R,
                                 ptr<int>(p.err), &extra));
            nl += extra;
        } else if (LL.n_up > 0) {   // c = Sigma^+ U^T chk; the K range split over z on small levels (cu is zeroed)
            constexpr int RMd = ApplyShape<double>::RM, CNd = ApplyShape<double>::CN;
            const int tiles = (int)(nbk(LL.n_up, 16 * CNd) * nbk(p.ops[l].rank, 16 * RMd));
            const int nz = std::max(1, std::min(16, std::min((S + AP_TK - 1) / AP_TK, (2 * p.num_sms + tiles - 1) / tiles)));
            RUN(launch_apply<double>(st, ptr<double>(p.ops[l].G1), S, p.ops[l].rank, S, ptr<int32_t>(LL.upb),
                                     ptr<int32_t>(LL.upb), 0, LL.n_up, ptr<double>(p.chk), S, cu, R, 0, 1, 0, nullptr,
                                     nz, 0, &p.apply_part, &nl));
        }
    }
    mark(p, 3);
    // ---- M2L in coefficients (Eq. (m2l))
    const T* c = nullptr;
    if (mixed) {
        // the FP32 copy of c feeds the SIMT M2L and the W lists only
        if (!p.m2l_tensor || p.lists[2].len > 0) {
            int64_t m = (int64_t)t.nboxes * R;
            k_to_f32<<<nbk(m, 256), 256, 0, st>>>(cu, ptr<float>(p.cu32), m);
            KF_LAUNCH();
            ++nl;
        }
        c = reinterpret_cast<const T*>(ptr<float>(p.cu32));
        if (p.m2l_tensor) {
            KF_TRY(m2l_tc_split(st, cu, t.nboxes, R, p.chi.p, p.clo.p, ptr<int>(p.cexp)));
            ++nl;
        }
    } else {
        c = reinterpret_cast<const T*>(cu);
    }
    if (sizeof(T) == 4 && p.m2l_tensor) {
        M2LTables tabs{};
        for (int l = 2; l < L; ++l) {
            tabs.hi[l] = p.ops[l].Thi.p;
            tabs.lo[l] = p.ops[l].Tlo.p;
            tabs.sT[l] = p.ops[l].tc_sT;
        }
        if (p.near_pending) KF_CUDA(cudaEventRecord(p.near_ev[0], st));   // (the near sums need q alone)
        KF_TRY(launch_m2l_tc(st, tabs, R, ptr<int4>(p.tc_tiles), p.tc_ntiles, ptr<int32_t>(p.tc_boxes),
                             ptr<int32_t>(p.vtab), ptr<int32_t>(p.tc_slots), p.chi.p, p.clo.p, ptr<int>(p.cexp),
                             reinterpret_cast<float*>(dd), ptr<int>(p.err)));
        ++nl;
        if (p.near_pending) KF_TRY(near_fork_launch(p, nl));
    } else {
        for (int l = 2; l < L; ++l) {
            auto& LL = p.lv[l];
            if (LL.n_tiles == 0) continue;
            dim3 g(LL.n_tiles, nbk(R, M2L_TM));
            k_m2l<T><<<g, 256, 0, st>>>(sel<T>(p.ops[l].T, p.ops[l].T32), R, ptr<int32_t>(p.vtab),
                                        ptr<int32_t>(LL.m2l_slots), t.level_start[l], t.level_start[l + 1], c, dd);
            KF_LAUNCH();
            ++nl;
        }
    }
    mark(p, 4);
    // ---- downward: S2L from the X list, L2L (Eq. (l2l)), then phi^d = U Sigma^+ d (Eq. (s2l))
    for (int l = 2; l < L; ++l) {
        auto& LL = p.lv[l];
        const LevelOps& op = p.ops[l];
        if (LL.n_x > 0) {   // Chebyshev: the values at B's nodes add straight into d
            k_s2l_x<(sizeof(T) == 4), T><<<LL.n_x, P2M_T, 0, st>>>(E, ptr<int32_t>(LL.xboxes), ptr<int32_t>(p.lists[3].off),
                                                                  ptr<int32_t>(p.lists[3].items), ptr<double>(p.q),
                                                                  p.cheb ? dd : ptr<T>(p.chkx), p.cheb ? R : S,
                                                                  p.cheb ? 1 : 0);
            KF_LAUNCH();
            ++nl;
            if (!p.cheb)
                RUN(launch_apply<T>(st, sel<T>(op.Vt, op.Vt32), S, op.rank, S, ptr<int32_t>(LL.xboxes),
                                    ptr<int32_t>(LL.xboxes), 0, LL.n_x, ptr<T>(p.chkx), S, dd, R, 1));
        }
        if (l >= 3) {
            auto& LP = p.lv[l - 1];
            const LevelOps& pop = p.ops[l - 1];
            if (LP.l2l_max > 0 && p.cheb) {   // Chebyshev: three 1-D passes per child
                const int64_t lo = t.level_start[l], cnt = t.level_start[l + 1] - lo;
                k_cheb_l2l_kron<T><<<(unsigned)cnt, KR_T, 0, st>>>(lo, ptr<int32_t>(t.parent), ptr<int32_t>(t.anchor),
                                                                   ptr<double>(p.cheb_A), p.m0, dd, R);
                KF_LAUNCH();
                ++nl;
            } else if (LP.l2l_max > 0 && sizeof(T) == 4 && p.l2l_tc && p.tc_count[l] >= p.tc_min_tiles) {
                // tensor cores: the parents' d split into FP16 hi / lo (the M2L operand buffers, free
                // by now), one slot per child octant, added onto the children's d
                const int64_t lo = t.level_start[l - 1], cnt = t.level_start[l] - lo;
                KF_TRY(m2l_tc_split_f32(st, reinterpret_cast<const float*>(dd) + lo * R, cnt, R,
                                        static_cast<char*>(p.chi.p) + lo * R * 2, static_cast<char*>(p.clo.p) + lo * R * 2,
                                        ptr<int>(p.cexp) + lo));
                ++nl;
                M2LTables tabs{};
                tabs.hi[l] = pop.Lhi.p;
                tabs.lo[l] = pop.Llo.p;
                tabs.sT[l] = pop.l2l_sT;
                RUN(launch_tc_translate(st, tabs, R, ptr<int4>(p.tc_tiles) + p.tc_first[l], p.tc_count[l],
                                        ptr<int32_t>(p.tc_boxes), ptr<int32_t>(p.ptab), 8,
                                        ptr<int32_t>(p.l2l_slots) + (int64_t)p.tc_first[l] * kSlotStride, p.chi.p,
                                        p.clo.p, ptr<int>(p.cexp), reinterpret_cast<float*>(dd), 1, ptr<int>(p.err)));
            } else if (LP.l2l_max > 0 && sizeof(T) == 4 && op.rank <= MM_TM && pop.rank <= MM_NS * MM_TK) {
                // FP32, one block per (octant, tile of parents), every chunk loaded at once (32
                // parents a tile where that gives every SM two blocks, else 16)
                auto* fn = 8 * nbk(LP.l2l_max, 32) >= 2u * p.num_sms ? launch_l2l_f32<32> : launch_l2l_f32<16>;
                KF_TRY(fn(st, ptr<float>(pop.Lo32), R, op.rank, pop.rank, ptr<int32_t>(LP.l2l_src),
                          ptr<int32_t>(LP.l2l_dst), ptr<int32_t>(LP.l2l_off), (int)LP.l2l_max,
                          reinterpret_cast<const float*>(dd), reinterpret_cast<float*>(dd)));
                ++nl;
            } else if (LP.l2l_max > 0)   // one launch, batched over the 8 child octants
                RUN(launch_apply<T>(st, sel<T>(pop.Lo, pop.Lo32), R, op.rank, pop.rank, ptr<int32_t>(LP.l2l_src),
                                    ptr<int32_t>(LP.l2l_dst), 0, LP.l2l_max, dd, R, dd, R, 1, 1, 0,
                                    ptr<int32_t>(LP.l2l_off), 8, (int64_t)R * R));
        }
        if (LL.n_leaf > 0 && !p.cheb && !(p.lat_far && l == p.nf_level))   // (lattice leaves: L2P reads d)
            RUN(launch_apply<T>(st, sel<T>(op.Ub, op.Ub32), R, S, op.rank, ptr<int32_t>(LL.leafs), ptr<int32_t>(LL.leafs), 0,
                                LL.n_leaf, dd, R, phid, S, 0));
    }
    // upward equivalent densities phi^u = V c for the W list (Chebyshev: the W list reads c)
    if (p.phiu.p && !p.cheb) {
        for (int l = 2; l < L; ++l) {
            const LevelOps& op = p.ops[l];
            RUN(launch_apply<T>(st, sel<T>(op.Vb, op.Vb32), R, S, op.rank, nullptr, nullptr, t.level_start[l],
                                (int)(t.level_start[l + 1] - t.level_start[l]), c, R, ptr<T>(p.phiu), S, 0));
        }
    }
#undef RUN
    return KIFMM_OK;
}

// q = I h^3 and I in sorted order (used by the surrogate's judge)
int kifmm_scatter_weights(Plan& p, const double* I, cudaStream_t st) {
    const int64_t n = p.tree.n;
    k_scatter_q<double><<<nbk(n, 256), 256, 0, st>>>(I, ptr<int32_t>(p.tree.perm), ptr<double>(p.w), n,
                                                            p.n_real, ptr<double>(p.Isort), ptr<double>(p.q));
    KF_LAUNCH();
    return KIFMM_OK;
}

int run_eval(Plan& p, const void* I, void* S_out, int dtype, double C) {
    int64_t nl = 0;   // kernels launched by this evaluation
    Tree& t = p.tree;
    cudaStream_t st = p.stream;
    const int64_t n = t.n;
    const bool mixed = p.precision == KIFMM_MIXED;
    EvalView E = make_view(p);
    mark(p, 0);
    if (dtype == KIFMM_F64)
        k_scatter_q<double><<<nbk(n, 256), 256, 0, st>>>((const double*)I, ptr<int32_t>(t.perm), ptr<double>(p.w),
                                                         n, p.n_real, ptr<double>(p.Isort), ptr<double>(p.q));
    else
        k_scatter_q<float><<<nbk(n, 256), 256, 0, st>>>((const float*)I, ptr<int32_t>(t.perm), ptr<double>(p.w),
                                                        n, p.n_real, ptr<double>(p.Isort), ptr<double>(p.q));
    KF_LAUNCH();
    ++nl;
    // the near sums (tensor-core lattice near field) read only q: they run on their own stream
    // beside the far field and are joined before the output combination. They are forked where
    // the M2L starts (the far field's run_far issues them after its M2L launch), so that the
    // earlier-issued M2L takes the SMs first and the near sums fill its last wave and the
    // downward pass; without a far field, right here.
    const bool fork = mixed && p.near_tc && p.near_st;
    p.near_forked = false;
    p.near_pending = fork && t.nlevels > 2 && !p.near_fork_early;
    if (fork && !p.near_pending) {
        KF_CUDA(cudaEventRecord(p.near_ev[0], st));
        const int rc = near_fork_launch(p, nl);
        if (rc != KIFMM_OK) {
            if (p.near_forked) cudaStreamWaitEvent(st, p.near_ev[1], 0);
            return rc;
        }
    }
    mark(p, 1);
    int far_rc = KIFMM_OK;
    if (t.nlevels > 2) {
        far_rc = mixed ? run_far<float>(p, E, nl) : run_far<double>(p, E, nl);
    } else {
        mark(p, 2);
        mark(p, 3);
        mark(p, 4);
    }
    if (far_rc == KIFMM_OK && p.near_pending) {   // (the SIMT M2L path: after the far field)
        KF_CUDA(cudaEventRecord(p.near_ev[0], st));
        far_rc = near_fork_launch(p, nl);
    }
    p.near_pending = false;
    if (far_rc != KIFMM_OK) {
        if (p.near_forked) cudaStreamWaitEvent(st, p.near_ev[1], 0);   // (a capture needs its fork joined)
        return far_rc;
    }
    mark(p, 5);
    // ---- targets: local expansion and W list, then the near field, self term and output
    if (p.nleaves > 0) {
        const int32_t* wo = ptr<int32_t>(p.lists[2].off);
        const int32_t* wi = ptr<int32_t>(p.lists[2].items);
        // Chebyshev: the W list reads the node weights c (stride R) and the local part
        // interpolates d in a second kernel
        if (p.lat_far && !p.cheb && t.nlevels > 2) {   // uniform lattice, no W list: the local part is one matrix from d
            KF_TRY(lat_l2p(p));
            if (p.lat_l2p_tc) ++nl;   // (the split of d, then the translation kernel)
        } else if (mixed) {
            auto* kl2p = p.far_series ? k_l2p<true, true, float> : k_l2p<true, false, float>;
            kl2p<<<(unsigned)p.nleaves, L2P_T, 0, st>>>(E, ptr<int32_t>(p.leaves), wo, wi, ptr<float>(p.phid),
                                                        p.cheb ? ptr<float>(p.cu32) : ptr<float>(p.phiu),
                                                        ptr<double>(p.far));
        } else {
            k_l2p<false, true, double><<<(unsigned)p.nleaves, L2P_T, 0, st>>>(
                E, ptr<int32_t>(p.leaves), wo, wi, ptr<double>(p.phid), p.cheb ? ptr<double>(p.cu) : ptr<double>(p.phiu),
                ptr<double>(p.far));
        }
        KF_LAUNCH();
        ++nl;
        if (p.cheb && t.nlevels > 2) {   // (on a lattice the 512-row matrix kernel was slower than this)
            if (mixed)
                k_l2p_cheb<true, float><<<(unsigned)p.nleaves, L2P_T, 0, st>>>(E, ptr<int32_t>(p.leaves), ptr<float>(p.dd),
                                                                              p.R, ptr<double>(p.far));
            else
                k_l2p_cheb<false, double><<<(unsigned)p.nleaves, L2P_T, 0, st>>>(E, ptr<int32_t>(p.leaves),
                                                                                ptr<double>(p.dd), p.R, ptr<double>(p.far));
            KF_LAUNCH();
            ++nl;
        }
    }
    mark(p, 6);
    if (mixed && p.near_tc) {   // uniform lattice: near field as per-offset contractions on the tensor cores
        if (p.near_forked) KF_CUDA(cudaStreamWaitEvent(st, p.near_ev[1], 0));   // join
        else KF_TRY(near_tc_contract(p, st, nl));
        KF_TRY(near_tc_finish(p, ptr<double>(p.far), C, S_out, dtype, nl));
    } else {
        size_t smem = (size_t)(mixed ? P2Q_CHUNK : P2P_CHUNK) * 16;
        const int32_t* uo = ptr<int32_t>(p.lists[0].off);
        const int32_t* ui = ptr<int32_t>(p.lists[0].items);
        unsigned g = (unsigned)p.nleaves;
        if (mixed) {
            auto* kf64 = p.p2p_series ? k_p2p_mixed<true, double> : k_p2p_mixed<false, double>;
            auto* kf32 = p.p2p_series ? k_p2p_mixed<true, float> : k_p2p_mixed<false, float>;
            if (dtype == KIFMM_F64)
                kf64<<<g, P2Q_T, smem, st>>>(E, ptr<int32_t>(p.leaves), uo, ui, ptr<double>(p.q), ptr<double>(p.far),
                                             ptr<double>(p.sigma), ptr<double>(p.Isort), ptr<int32_t>(t.perm), C,
                                             (double*)S_out);
            else
                kf32<<<g, P2Q_T, smem, st>>>(E, ptr<int32_t>(p.leaves), uo, ui, ptr<double>(p.q), ptr<double>(p.far),
                                             ptr<double>(p.sigma), ptr<double>(p.Isort), ptr<int32_t>(t.perm), C,
                                             (float*)S_out);
        } else {
            if (dtype == KIFMM_F64)
                k_p2p<false, double><<<g, P2P_T, smem, st>>>(E, ptr<int32_t>(p.leaves), uo, ui, ptr<double>(p.q), ptr<double>(p.far),
                                                             ptr<double>(p.sigma), ptr<double>(p.Isort), ptr<int32_t>(t.perm), C, (double*)S_out);
            else
                k_p2p<false, float><<<g, P2P_T, smem, st>>>(E, ptr<int32_t>(p.leaves), uo, ui, ptr<double>(p.q), ptr<double>(p.far),
                                                            ptr<double>(p.sigma), ptr<double>(p.Isort), ptr<int32_t>(t.perm), C, (float*)S_out);
        }
        KF_LAUNCH();
        ++nl;
    }
    mark(p, 7);
    p.eval_launches = nl;
    return KIFMM_OK;
}

}  // namespace kifmm
