// Near field (Eq. (nearfar), first sum) on a uniform lattice, on the tensor cores.
//
// When every leaf is a full block of nc x nc x nc cells of one uniform grid (the same
// level for all leaves, cell centres on the lattice, the points of each leaf in the same
// local order), the contribution of a neighbour leaf A at offset delta (in {-1, 0, 1}^3)
// to the targets of B is one fixed matrix applied to A's weights:
//   near[B][i] += sum_j K_delta[i][j] q[A][j],  K_delta[i][j] = K(h |nc delta + c_j - c_i|),
// c_i the integer cell of local point i, and K_0[i][i] = 0 (the self term is added apart).
// Every pair of the U lists is still summed; only the kernel values, which depend on the
// geometry alone, are tabulated at plan time, like the far-field translation operators.
// The 27 matrices (R = nc^3 rows) go through the tensor-core translation kernel of M2L
// (FP16 x 3 split, per-offset FP32 accumulators), with the leaves' weight rows as its
// coefficient rows. Plans whose points are not such a lattice use the pair kernel.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>

#include "internal.cuh"
#include "kernel.cuh"

namespace kifmm {

static inline unsigned nbn(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// local cell index ix + nc (iy + nc iz) of every sorted point inside its leaf; *bad is set
// where a point is off the lattice (more than 1e-6 cells) or outside its leaf
__global__ void k_nf_local(const double* pts, const int32_t* leaf_of, const double* centre, int64_t n, double h,
                           double r, int nc, int32_t* lidx, int* bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int B = leaf_of[i];
    int idx[3];
    for (int k = 0; k < 3; ++k) {
        const double u = (pts[3 * i + k] - (centre[3 * (int64_t)B + k] - r)) / h - 0.5;
        const double ur = rint(u);
        idx[k] = (int)ur;
        if (fabs(u - ur) > 1e-6 || idx[k] < 0 || idx[k] >= nc) atomicOr(bad, 1);
    }
    lidx[i] = idx[0] + nc * (idx[1] + nc * idx[2]);
}

// every leaf: npl points, the k-th of them at local cell ref[k], at level lf, and leaf
// ordinal o holding the points o npl .. (o + 1) npl - 1
__global__ void k_nf_check(const int32_t* leaves, int64_t nleaves, const int32_t* pstart, const int32_t* pend,
                           const int32_t* level, int lf, int npl, const int32_t* lidx, const int32_t* ref, int* bad) {
    const int64_t o = blockIdx.x;
    if (o >= nleaves) return;
    const int B = leaves[o];
    if (threadIdx.x == 0 && (pend[B] - pstart[B] != npl || pstart[B] != o * npl || level[B] != lf)) atomicOr(bad, 1);
    if (pend[B] - pstart[B] != npl) return;
    for (int k = threadIdx.x; k < npl; k += blockDim.x)
        if (lidx[pstart[B] + k] != ref[k]) atomicOr(bad, 1);
}

// utab[o][slot]: ordinal of the neighbour leaf of leaf o at the offset slot (-1 if none);
// every member of U(B) must be a same-level box within one box of B
__global__ void k_nf_utab(const int32_t* leaves, int64_t nleaves, const int32_t* uoff, const int32_t* uitems,
                          const int32_t* anchor, const int32_t* level, const int32_t* pstart, int npl, int32_t* utab,
                          int* bad) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nleaves) return;
    const int B = leaves[o];
    utab[o * kOffsetSlots + 3 + 7 * 3 + 49 * 3] = (int32_t)o;   // the leaf itself (offset 0)
    for (int u = uoff[B]; u < uoff[B + 1]; ++u) {
        const int A = uitems[u];
        const int dx = anchor[3 * A] - anchor[3 * B], dy = anchor[3 * A + 1] - anchor[3 * B + 1],
                  dz = anchor[3 * A + 2] - anchor[3 * B + 2];
        if (level[A] != level[B] || abs(dx) > 1 || abs(dy) > 1 || abs(dz) > 1) {
            atomicOr(bad, 1);
            continue;
        }
        utab[o * kOffsetSlots + (dx + 3) + 7 * (dy + 3) + 49 * (dz + 3)] = pstart[A] / npl;
    }
}

// T[slot][i][j] = K(h |nc delta + c_j - c_i|) for the 27 near slots (zero on the diagonal of
// delta = 0); the other slots are left as they are (zero)
__global__ void k_nf_table(const int32_t* ref, int nc, int R, double h, KParams kp, double* T) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 27LL * R * R) return;
    const int d = (int)(e / ((int64_t)R * R)), i = (int)((e / R) % R), j = (int)(e % R);
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    const int ci = ref[i], cj = ref[j];
    const int ix = ci % nc, iy = (ci / nc) % nc, iz = ci / (nc * nc);
    const int jx = cj % nc, jy = (cj / nc) % nc, jz = cj / (nc * nc);
    const double ux = nc * dx + jx - ix, uy = nc * dy + jy - iy, uz = nc * dz + jz - iz;
    const int slot = (dx + 3) + 7 * (dy + 3) + 49 * (dz + 3);
    const double rr = h * sqrt(ux * ux + uy * uy + uz * uz);
    T[((int64_t)slot * R + i) * R + j] = rr > 0.0 ? kern_f64(rr, kp) : 0.0;
}

// S in the caller's order: C (near + far + sigma I)
template <class TO>
__global__ void k_nf_finish(const float* near, const double* far, const double* sigma, const double* Is,
                            const int32_t* perm, int64_t n, double C, TO* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[perm[i]] = (TO)(C * ((double)near[i] + far[i] + sigma[i] * Is[i]));
}

int near_tc_plan(Plan& p) {
    p.near_tc = false;
    const char* env = std::getenv("KIFMM_P2P");
    if (env && std::string(env) == "generic") return KIFMM_OK;
    Tree& t = p.tree;
    if (p.precision != KIFMM_MIXED || !(p.uniform_h > 0.0) || p.nleaves < 1) return KIFMM_OK;
    // the level of the first leaf; k_nf_check below requires every leaf on it
    int32_t first = 0, lf = 0;
    cudaStream_t st = p.stream;
    KF_CUDA(cudaMemcpyAsync(&first, p.leaves.p, 4, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    KF_CUDA(cudaMemcpyAsync(&lf, ptr<int32_t>(t.level) + first, 4, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    if (lf < 0 || lf > kMaxLevel) return KIFMM_OK;
    const double h = p.uniform_h, r = t.side / (double)(2ll << lf);
    const int nc = (int)std::lround(2.0 * r / h);
    if (nc < 1 || std::fabs(nc * h - 2.0 * r) > 1e-9 * 2.0 * r) return KIFMM_OK;
    const int npl = nc * nc * nc, R = npl;
    if (R % 32 != 0 || !m2l_tc_supported(R) || (int64_t)npl * p.nleaves != t.n) return KIFMM_OK;
    const int64_t n = t.n, nl = p.nleaves;
    DevBuf lidx, ref, bad;
    KF_TRY(dev_alloc(lidx, n * 4));
    KF_TRY(dev_alloc(ref, npl * 4));
    KF_TRY(dev_alloc(bad, 4));
    KF_CUDA(cudaMemsetAsync(bad.p, 0, 4, st));
    k_nf_local<<<nbn(n, 256), 256, 0, st>>>(ptr<double>(p.pts), ptr<int32_t>(p.leaf_of), ptr<double>(t.centre), n, h,
                                             r, nc, ptr<int32_t>(lidx), ptr<int>(bad));
    KF_LAUNCH();
    // the local order of the first leaf is the reference; it must be a permutation of the cells
    int32_t p0 = 0;
    KF_CUDA(cudaMemcpyAsync(&p0, ptr<int32_t>(t.pstart) + first, 4, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    auto release = [&]() {
        for (DevBuf* d : {&lidx, &ref, &bad}) dev_free(*d);
    };
    if (p0 != 0) {   // then the first leaf holds points 0 .. npl - 1 (npl nleaves = n)
        release();
        return KIFMM_OK;
    }
    std::vector<int32_t> href(npl);
    KF_CUDA(cudaMemcpyAsync(href.data(), lidx.p, npl * 4, cudaMemcpyDeviceToHost, st));
    int hbad = 0;
    KF_CUDA(cudaMemcpyAsync(&hbad, bad.p, 4, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    if (hbad) {
        release();
        return KIFMM_OK;
    }
    {
        std::vector<char> seen(npl, 0);
        for (int k = 0; k < npl; ++k) {
            if (href[k] < 0 || href[k] >= npl || seen[href[k]]) {
                release();
                return KIFMM_OK;
            }
            seen[href[k]] = 1;
        }
    }
    KF_CUDA(cudaMemcpyAsync(ref.p, href.data(), npl * 4, cudaMemcpyHostToDevice, st));
    k_nf_check<<<(unsigned)nl, 128, 0, st>>>(ptr<int32_t>(p.leaves), nl, ptr<int32_t>(t.pstart), ptr<int32_t>(t.pend),
                                              ptr<int32_t>(t.level), lf, npl, ptr<int32_t>(lidx), ptr<int32_t>(ref),
                                              ptr<int>(bad));
    KF_LAUNCH();
    KF_TRY(dev_alloc(p.nf_utab, (size_t)nl * kOffsetSlots * 4));
    KF_CUDA(cudaMemsetAsync(p.nf_utab.p, 0xFF, (size_t)nl * kOffsetSlots * 4, st));
    k_nf_utab<<<nbn(nl, 128), 128, 0, st>>>(ptr<int32_t>(p.leaves), nl, ptr<int32_t>(p.lists[0].off),
                                             ptr<int32_t>(p.lists[0].items), ptr<int32_t>(t.anchor),
                                             ptr<int32_t>(t.level), ptr<int32_t>(t.pstart), npl,
                                             ptr<int32_t>(p.nf_utab), ptr<int>(bad));
    KF_LAUNCH();
    KF_CUDA(cudaMemcpyAsync(&hbad, bad.p, 4, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    if (hbad) {
        dev_free(p.nf_utab);
        release();
        return KIFMM_OK;
    }
    // the 27 near-offset matrices, FP64, then their FP16 hi / lo images for the tensor cores
    DevBuf T;
    const int64_t RR = (int64_t)R * R;
    KF_TRY(dev_alloc(T, kOffsetSlots * RR * 8));
    KF_CUDA(cudaMemsetAsync(T.p, 0, kOffsetSlots * RR * 8, st));
    k_nf_table<<<nbn(27 * RR, 256), 256, 0, st>>>(ptr<int32_t>(ref), nc, R, h, make_kparams(p.a, p.b), ptr<double>(T));
    KF_LAUNCH();
    KF_TRY(dev_alloc(p.nf_Thi, (size_t)m2l_tc_table_elems(R) * 2));
    KF_TRY(dev_alloc(p.nf_Tlo, (size_t)m2l_tc_table_elems(R) * 2));
    KF_TRY(m2l_tc_prepare(st, ptr<double>(T), R, p.nf_Thi.p, p.nf_Tlo.p, &p.nf_sT));
    // tiles of 128 leaves (ordinals), every tile over the 27 near slots
    const int ntiles = (int)((nl + 127) / 128);
    std::vector<int4> tiles(ntiles);
    for (int k = 0; k < ntiles; ++k) tiles[k] = make_int4(lf, 128 * k, (int)std::min<int64_t>(128, nl - 128LL * k), 0);
    std::vector<int32_t> slots((size_t)ntiles * kSlotStride, 0), ids(nl);
    for (int k = 0; k < ntiles; ++k) {
        int32_t* s = slots.data() + (size_t)k * kSlotStride;
        s[0] = 27;
        int c = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) s[1 + c++] = (dx + 3) + 7 * (dy + 3) + 49 * (dz + 3);
    }
    for (int64_t o = 0; o < nl; ++o) ids[o] = (int32_t)o;
    KF_TRY(dev_alloc(p.nf_tiles, tiles.size() * sizeof(int4)));
    KF_TRY(dev_alloc(p.nf_slots, slots.size() * 4));
    KF_TRY(dev_alloc(p.nf_boxes, ids.size() * 4));
    KF_CUDA(cudaMemcpyAsync(p.nf_tiles.p, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    KF_CUDA(cudaMemcpyAsync(p.nf_slots.p, slots.data(), slots.size() * 4, cudaMemcpyHostToDevice, st));
    KF_CUDA(cudaMemcpyAsync(p.nf_boxes.p, ids.data(), ids.size() * 4, cudaMemcpyHostToDevice, st));
    KF_TRY(dev_alloc(p.nf_qhi, (size_t)n * 2));
    KF_TRY(dev_alloc(p.nf_qlo, (size_t)n * 2));
    KF_TRY(dev_alloc(p.nf_qexp, (size_t)nl * 4));
    KF_TRY(dev_alloc(p.nf_near, (size_t)n * 4));
    KF_CUDA(cudaStreamSynchronize(st));
    dev_free(T);
    release();
    p.nf_R = R;
    p.nf_level = lf;
    p.nf_ntiles = ntiles;
    p.near_tc = true;
    return KIFMM_OK;
}

int near_tc_eval(Plan& p, const double* far, double C, void* out, int dtype, int64_t& nl) {
    cudaStream_t st = p.stream;
    const int64_t n = p.tree.n;
    KF_TRY(m2l_tc_split(st, ptr<double>(p.q), p.nleaves, p.nf_R, p.nf_qhi.p, p.nf_qlo.p, ptr<int>(p.nf_qexp)));
    ++nl;
    M2LTables tabs{};
    tabs.hi[p.nf_level] = p.nf_Thi.p;
    tabs.lo[p.nf_level] = p.nf_Tlo.p;
    tabs.sT[p.nf_level] = p.nf_sT;
    KF_TRY(launch_m2l_tc(st, tabs, p.nf_R, ptr<int4>(p.nf_tiles), p.nf_ntiles, ptr<int32_t>(p.nf_boxes),
                         ptr<int32_t>(p.nf_utab), ptr<int32_t>(p.nf_slots), p.nf_qhi.p, p.nf_qlo.p, ptr<int>(p.nf_qexp),
                         ptr<float>(p.nf_near), ptr<int>(p.err)));
    ++nl;
    if (dtype == KIFMM_F64)
        k_nf_finish<double><<<nbn(n, 256), 256, 0, st>>>(ptr<float>(p.nf_near), far, ptr<double>(p.sigma),
                                                          ptr<double>(p.Isort), ptr<int32_t>(p.tree.perm), n, C,
                                                          (double*)out);
    else
        k_nf_finish<float><<<nbn(n, 256), 256, 0, st>>>(ptr<float>(p.nf_near), far, ptr<double>(p.sigma),
                                                         ptr<double>(p.Isort), ptr<int32_t>(p.tree.perm), n, C,
                                                         (float*)out);
    KF_LAUNCH();
    ++nl;
    return KIFMM_OK;
}

}  // namespace kifmm
