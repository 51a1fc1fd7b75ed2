// Internal declarations shared by the translation units of libkifmm.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/kifmm.h"

namespace kifmm {

constexpr int kKeyBits = 21;
constexpr int kMaxLevel = 20;
constexpr int kOffsetSlots = 343;   // (dx, dy, dz) in [-3, 3]^3
constexpr int kSlotStride = 344;    // per tensor-core translation tile: [count, slot_0, slot_1, ...]
// Default surface radii in box half-widths: upward equivalent / downward check at 1.05 r, upward
// check / downward equivalent at 2.95 r, the reading that reproduces the accuracy the paper reports
// at its own test sizes (Sec. 4); the schematic Fig. fmulloc draws 1.2 r and 2.6 r.
constexpr double kRInner = 1.05;
constexpr double kROuter = 2.95;
// Upward solves of levels with at most kOzMinBoxes boxes take the FP64-pipe GEMM with its K
// range split over many CTAs: a tensor-core slice-product CTA needs about 45 us, which a
// handful of CTAs cannot hide.
constexpr int kOzMinBoxes = 1024;
// Levels with fewer tensor-core tiles than this take the SIMT apply for M2M / L2L: a tile
// walks its slots one pipeline stage at a time (about 1.2 us a stage), so a launch of a few
// tiles costs about 29 us whatever its work.
constexpr int kTcMinTiles = 16;

// ---- error plumbing ---------------------------------------------------------------
void set_error(const std::string& msg);
struct Status {
    int code = KIFMM_OK;
    std::string msg;
};
#define KF_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            kifmm::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));        \
            return KIFMM_ERR_CUDA;                                                        \
        }                                                                                 \
    } while (0)
#define KF_LAUNCH()                                                                       \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess) {                                                          \
            kifmm::set_error(std::string("kernel launch (") + __FILE__ + ":" +            \
                             std::to_string(__LINE__) + "): " + cudaGetErrorString(e_));  \
            return KIFMM_ERR_CUDA;                                                        \
        }                                                                                 \
    } while (0)
#define KF_TRY(expr)                                                                      \
    do {                                                                                  \
        int s_ = (expr);                                                                  \
        if (s_ != KIFMM_OK) return s_;                                                    \
    } while (0)

// ---- device buffer owned by a plan ---------------------------------------------------
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};
int dev_alloc(DevBuf& b, size_t bytes);
// Scope of kifmm_plan in which KIFMM_FAIL_ALLOC=k fails the k-th device allocation (tests)
struct AllocFaultScope {
    AllocFaultScope();
    ~AllocFaultScope();
};
void dev_free(DevBuf& b);
template <class T> T* ptr(const DevBuf& b) { return reinterpret_cast<T*>(b.p); }

// ---- plan ---------------------------------------------------------------------------
struct Tree {
    int64_t n = 0;          // points
    int64_t nboxes = 0;
    int nlevels = 0;
    std::vector<int64_t> level_start;   // host copy, nlevels + 1 entries
    double origin[3] = {0, 0, 0};
    double side = 0;
    // device arrays
    DevBuf keys;      // u64[n] sorted Morton keys
    DevBuf perm;      // i32[n] input index of sorted point k
    DevBuf level;     // i32[nb]
    DevBuf anchor;    // i32[3*nb]
    DevBuf mcode;     // u64[nb] Morton code of the anchor at the box's level
    DevBuf parent;    // i32[nb]
    DevBuf child;     // i32[8*nb]
    DevBuf pstart;    // i32[nb]
    DevBuf pend;      // i32[nb]
    DevBuf leaf;      // i32[nb]
    DevBuf centre;    // f64[3*nb]
};

struct Csr {
    DevBuf off;    // i32[nb+1]
    DevBuf items;  // i32[len]
    int64_t len = 0;
};

struct LevelOps {
    int level = 0;
    double r = 0;        // box half-width
    int rank = 0;        // kept rank r of the truncated SVD of K(x^{B,u}, y^{B,u})
    // FP64 basis matrices, R = padded coefficient count (zero beyond the rank)
    DevBuf G1;           // [R][S] Sigma^+ U^T: upward check potential -> coefficients c
    DevBuf Vb;           // [S][R] V: coefficients c -> upward equivalent density
    DevBuf Ub;           // [S][R] U Sigma^+: coefficients d -> downward equivalent density
    DevBuf Vt;           // [R][S] V^T: downward check potential -> coefficients d
    DevBuf T;            // [343][R][R] M2L in coefficients, V^T K(x^{B,d}, y^{A,u}) V
    DevBuf Mc;           // [8][S][R] M2M to the parent's upward check surface, K(x^{P,u}, y^{C_o,u}) V_{l+1}
    DevBuf Lo;           // [8][R][R] L2L in coefficients, parent level = this level
    // FP32 copies (mixed form)
    DevBuf T32, Ub32, Vb32, Vt32, Lo32, Mc32;
    // tensor-core M2L operands: FP16 hi/lo of T 2^tc_sT, [slot][k-chunk][row][128-byte swizzled row]
    DevBuf Thi, Tlo;
    int tc_sT = 0;
    // tensor-core L2L (parent level = this level): FP16 hi/lo of Lo 2^l2l_sT, 8 slots
    DevBuf Lhi, Llo;
    int l2l_sT = 0;
    // tensor-core M2M translations (parent level = this level): FP16 hi/lo of Mc (rows padded to R)
    DevBuf Mhi, Mlo;
    int m2m_sT = 0;
    // FP64-exact upward solve on the tensor cores: integer slices of G1 (swizzled images) and
    // the per-row power-of-two exponents
    DevBuf ozG1, ozEr;
};

struct Plan {
    int precision = KIFMM_FP64;
    int self_mode = KIFMM_SELF_CELL_EXACT;
    double pinv_eps = 1e-5;
    double r_in = kRInner, r_out = kROuter;   // surface radii in box half-widths
    cudaStream_t stream = nullptr;
    double a = 0, b = 0;
    int m0 = 6, S = 152, Sp = 152, R = 32;   // R: padded coefficient count
    int leaf_size = 64;
    Tree tree;
    Csr lists[4];                 // U, V, W, X
    DevBuf vtab;                  // i32[nb * 343]: source box of V(B) at offset slot, -1 if none
    std::vector<LevelOps> ops;    // indexed by level (entries below 2 unused)
    DevBuf surf;                  // f64[3*S] unit lattice (Chebyshev representation: the p^3 nodes)
    DevBuf ctab, ctab32;          // f64 / f32 [p][10]: c_k T_k(node_n), c_0 = 1/p, c_k = 2/p (Chebyshev only)
    DevBuf cheb_A;                // f64 [2][p][p]: 1-D factors of the M2M / L2L interpolation (Chebyshev only)
    // per-point data in sorted order
    DevBuf pts;       // f64[3n] sorted coordinates
    DevBuf loc32;     // f32[4n] coordinates relative to the leaf centre (x, y, z, pad)
    DevBuf w;         // f64[n] cell volume h^3
    DevBuf sigma;     // f64[n] self-cell value
    DevBuf leaf_of;   // i32[n] leaf box of each sorted point
    // leaves and per-level box lists
    DevBuf leaves;    // i32[nleaves]
    int64_t nleaves = 0;
    DevBuf p2m_boxes;      // i32: leaves of level >= 2
    int64_t n_p2m = 0;
    // eval workspace (T = f64 in the FP64 form, f32 in the mixed form)
    DevBuf q;          // f64[n]  I*h^3 (sorted)
    DevBuf Isort;      // f64[n]
    DevBuf chk;        // f64[nb*S] upward check potentials of the leaves (S2M)
    DevBuf chkx;       // T[nb*S]  downward check potentials from the X list (S2L)
    DevBuf cu;         // f64[nb*R] upward coefficients c
    DevBuf cu32;       // f32[nb*R] (mixed) FP32 copy of c for the SIMT M2L and the W list
    DevBuf chi, clo;   // f16[nb*R] (mixed, tensor-core M2L) hi/lo parts of c 2^cexp
    DevBuf cexp;       // i32[nb] per-box power-of-two scale of chi/clo
    DevBuf dd;         // T[nb*R]  downward coefficients d
    DevBuf phid;       // T[nb*S]  downward equivalent densities of the leaves
    DevBuf phiu;       // T[nb*S]  upward equivalent densities (only when W lists exist)
    DevBuf far;        // f64[n] far-field part at the sorted points
    DevBuf host_I;     // staging for kifmm_eval_host (n * 8 bytes each)
    DevBuf host_S;
    // per-level work lists for the batched matrix applications
    struct LevelLists {
        DevBuf all;        int n_all = 0;        // boxes of the level
        DevBuf leafs;      int n_leaf = 0;       // leaves of the level
        DevBuf nonleaf;    int n_nonleaf = 0;    // non-leaf boxes of the level
        DevBuf m2m_src[8]; DevBuf m2m_dst[8]; int n_m2m[8] = {0};   // child (src), parent (dst)
        DevBuf m2l_tiles;  int n_tiles = 0;      // tile -> first box (tiles of kM2LTile boxes)
        DevBuf m2l_slots;  DevBuf m2l_slot_off;  // per tile: list of active offset slots
        DevBuf m2l_boxes;                          // boxes of the level grouped by octant (tensor-core M2L)
        DevBuf m2l_slots128; int n_tiles128 = 0;  // active offset slots per tile of 128 grouped boxes
        DevBuf xboxes;     int n_x = 0;          // boxes with non-empty X list
        DevBuf parents;    int n_par = 0;        // non-leaf boxes of the level
        DevBuf par_kids;                         // [8][n_par] child per octant, -1 if empty
        DevBuf upb;        int n_up = 0;         // leaves then parents of the level (upward solves)
        DevBuf l2l_src, l2l_dst, l2l_off;        // (parent, child) pairs concatenated over octants
        int l2l_max = 0;                         // largest octant batch
    };
    std::vector<LevelLists> lv;
    DevBuf wleaves;   int n_wleaves = 0;      // leaves with non-empty W list
    int64_t eval_launches = 0;   // kernels of the last evaluation
    bool m2l_tensor = false;     // M2L on tcgen05 (mixed form)
    bool l2l_tc = false;         // L2L through the same kernel (mixed form)
    DevBuf ptab, l2l_slots;      // i32[nb][8] parent at the box's octant slot; per-tile L2L slot lists
    int tc_first[kMaxLevel + 1] = {0}, tc_count[kMaxLevel + 1] = {0};   // M2L tiles of each level
    bool m2m_tc = false;         // M2M translations through the same kernel (mixed form)
    DevBuf m2m_tiles, m2m_slots, stage32;   // parent tiles per level, their 8 slots, FP32 staging [nb][m2m_R]
    DevBuf apply_part;                      // partial sums of the SIMT applies split over their terms
    int m2m_R = 0;                          // square table size of the M2M translations: max(S, R) rounded to 32
    DevBuf m2m_hi, m2m_lo;                  // children's c split FP16 x 2 in rows of m2m_R (when m2m_R > R)
    int m2m_first[kMaxLevel + 1] = {0}, m2m_count[kMaxLevel + 1] = {0};
    int num_sms = 1;             // multiprocessors of the plan's device (grid sizing)
    bool p2p_series = true;      // some near pair is closer than 0.5 / (b - a) (mixed P2P)
    bool cheb = false;           // Chebyshev-node representation (p = m0, S = p^3), no pseudo-inverses
    double uniform_h = 0;        // cell edge of a uniform-h plan (0: per-point h, or rectangular cells)
    int64_t n_real = 0;          // the caller's points; tree.n - n_real zero-weight padding cells follow them
    int kind = 0;                // kernel: 0 the paper's, 1 three-exponential Helmholtz, 2 three-group
    bool rect = false;           // every cell is the rectangular box cell_dims (hx, hy, hz)
    double cell_dims[3] = {0, 0, 0};
    // near field on the tensor cores (mixed form, uniform lattice; near_tc.cu)
    bool near_tc = false;
    int nf_R = 0, nf_level = 0, nf_sT = 0, nf_ntiles = 0;
    DevBuf nf_utab, nf_Thi, nf_Tlo, nf_tiles, nf_slots, nf_boxes, nf_qhi, nf_qlo, nf_qexp, nf_near, nf_ref;
    bool lat_far = false;        // S2M and local L2P on the same lattice (surface form, no W / X lists)
    DevBuf lat_P;                // f32 [S][npl + 1]: K between the leaf's check surface and its cells
    DevBuf lat_Q;                // f32 [R][npl + 1]: P^T Ub, the leaf's local expansion from its coefficients d
    bool lat_l2p_tc = false;     // that expansion through the tensor-core kernel (FP32 rows in lat_fst)
    DevBuf lat_Thi, lat_Tlo, lat_iota, lat_slots, lat_fst;
    int lat_sT = 0;
    bool lat_up = false;         // leaves' c = (G1 P) q on the tensor cores, FP64-exact (no leaf S2M)
    DevBuf lat_Mimg, lat_Mer;    // slice image and row exponents of M = G1 P (rank x npl)
    bool far_series = true;      // likewise for a leaf's points and its check / equivalent surfaces
    bool oz = false;             // upward pseudo-inverse by exact slicing on the tensor cores (mixed form)
    DevBuf ozBox, ozEb;          // per-level work space: box slice images, box exponents
    int oz_min = kOzMinBoxes;    // levels with more upward solves than this use the slice products
    int tc_min_tiles = kTcMinTiles;   // levels with at least this many tiles: tensor-core M2M / L2L
    DevBuf tc_tiles;             // int4 per tile: level, first box in tc_boxes, box count, 0
    DevBuf tc_boxes;             // boxes of every level grouped by octant, level after level
    DevBuf tc_slots;             // [tile][344] active offset slots
    int tc_ntiles = 0;
    DevBuf err;                  // int: device-side error code (bounded waits)
    int64_t p2p_pairs = 0;       // near-field pairs of one evaluation
    double m2l_flops = 0;        // algorithmic M2L flop of one evaluation (2 r^2 per V pair)
    double up_flops = 0;         // FP64 upward flop (projection 2 r S per leaf, M2M 2 r r' per child)
    // timing
    bool timing = false;
    cudaEvent_t ev[9] = {};
    uint64_t nvtx_range = 0;     // open NVTX range of the current phase (0: none)
    float phase_ms[8] = {0};
    int n_phases = 0;
    // batch graph, keyed on the batch's arguments (plan ids, buffers, count, dtype, lanes, C bits)
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<uint64_t> graph_key;
    uint64_t uid = 0;            // process-wide unique id of this plan (never reused)
    // concurrent batch lanes owned by this plan: streams, and events [0] fork, [1 + j] join
    std::vector<cudaStream_t> lanes;
    std::vector<cudaEvent_t> lane_ev;
    // the near-field contraction's own stream (tensor-core lattice near field): it needs only
    // the sorted weights, so it runs beside the far field; events [0] fork, [1] join
    cudaStream_t near_st = nullptr;
    cudaEvent_t near_ev[2] = {nullptr, nullptr};
    cudaEvent_t near_tev[2] = {nullptr, nullptr};   // its start and end (phase timing)
    bool near_forked = false;    // the last evaluation ran the near sums on near_st
    bool near_pending = false;   // (during an evaluation) the far field is to fork them at its M2L
    bool near_fork_early = false;   // fork them after the weights' scatter instead (KIFMM_NEAR_STREAM=early)
};

// tree.cu
// the full grid of a box of cubic cells (edge h) padded with zero-weight cells to extents that
// are multiples of 2 nc, after the caller's n points (out, *n_total > n; nothing allocated when
// the extents already are), and the root cube at the grid's corner with side nc h 2^L in
// root[0..3]; other point sets: *n_total = n, root[3] = 0
int pad_to_lattice(cudaStream_t st, const double* pts, int64_t n, double h, int nc, DevBuf& out, int64_t* n_total,
                   double root[4]);
int build_tree(Plan& p, const double* points_dev, const double* h_dev, double uniform_h,
               const kifmm_opts& o);
int build_lists(Plan& p);
int radix_sort_pairs(uint64_t* keys, int32_t* vals, int64_t n, int key_bits, cudaStream_t st,
                     DevBuf& tmp_keys, DevBuf& tmp_vals, DevBuf& hist);
int device_scan_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total_host,
                    cudaStream_t st, DevBuf& scratch);
// operators.cu
int build_operators(Plan& p);
int build_self_terms(Plan& p, const double* h_dev, double uniform_h);
// m2l_tc.cu
int m2l_tc_supported(int R);
int64_t m2l_tc_table_elems(int R, int nslots = kOffsetSlots);   // FP16 elements of one level's Thi (or Tlo)
int m2l_tc_prepare(cudaStream_t st, const double* T, int R, void* Thi, void* Tlo, int* sT_out,
                   int nslots = kOffsetSlots);
int m2l_tc_split(cudaStream_t st, const double* c, int64_t nb, int R, void* chi, void* clo, int* cexp);
// the same with output rows of ldo >= R halves (columns R..ldo-1 zero)
int m2l_tc_split_pad(cudaStream_t st, const double* c, int64_t nb, int R, int ldo, void* chi, void* clo, int* cexp);
int m2l_tc_split_f32(cudaStream_t st, const float* c, int64_t nb, int R, void* chi, void* clo, int* cexp);
struct M2LTables {                 // per-level FP16 hi/lo M2L tables for the tensor-core kernel
    const void* hi[kMaxLevel + 1];
    const void* lo[kMaxLevel + 1];
    int sT[kMaxLevel + 1];         // the tables hold T 2^sT
};
int launch_m2l_tc(cudaStream_t st, const M2LTables& tabs, int R, const int4* tiles, int ntiles, const int32_t* boxes,
                  const int32_t* vtab, const int32_t* slots, const void* chi, const void* clo, const int* cexp, float* d,
                  int* err);
// the same kernel with any source table stride (nslots slots per target box) and, with
// accum != 0, the result added to d (L2L onto the M2L result)
int launch_tc_translate(cudaStream_t st, const M2LTables& tabs, int R, const int4* tiles, int ntiles,
                        const int32_t* boxes, const int32_t* vtab, int vstride, const int32_t* slots, const void* chi,
                        const void* clo, const int* cexp, float* d, int accum, int* err);
// near_tc.cu: near field on a uniform lattice
int near_tc_plan(Plan& p);
int near_tc_contract(Plan& p, cudaStream_t st, int64_t& nl);   // the near sums into nf_near on st
int near_tc_finish(Plan& p, const double* far, double C, void* out, int dtype, int64_t& nl);
int lat_s2m(Plan& p);   // chk of every leaf (lat_far plans)
int lat_l2p(Plan& p);   // far of every point from the leaves' d (lat_far plans)
int lat_up_plan(Plan& p);   // M = G1 P for the leaves' FP64-exact upward solve (after the slice set-up)
int lat_up_apply(Plan& p, double* cu, int64_t& nl);   // c of every leaf = M q
// pinv_oz.cu: FP64-exact c = Sigma^+ U^T chk on the tensor cores
int pinv_oz_supported(int S);
size_t pinv_oz_op_bytes(int S, int rank);
size_t pinv_oz_box_bytes(int S, int n);
double pinv_oz_mma_flops(int S, int rank, int n);   // tensor-core flop of one level's solve
int pinv_oz_prepare(cudaStream_t st, const double* G1, int S, int rank, void* img, int* er);
// c[boxes[p]] = Op chk[in_rows ? in_rows[p] : boxes[p]] for p < n (rows of chk have S entries)
int pinv_oz_apply(cudaStream_t st, const double* chk, int S, const int32_t* boxes, const int32_t* in_rows, int n,
                  const void* opimg, const int* er, int rank, void* bimg, int* eb, double* cu, int R, int* err,
                  int64_t* launches);
// tune.cu: targets drawn in proportion to a field (probability 0.5 |S_i| / sum |S| + 0.5 / n,
// systematic sampling, weights 1 / (k m_i)); perm (sorted -> caller) gives sorted indices
size_t importance_ws_bytes(int64_t n, int k);
int importance_targets(cudaStream_t st, const double* S, int64_t n, int k, uint64_t seed, const int32_t* perm,
                       int64_t nperm, void* ws, int32_t* tcaller, int32_t* tsorted, double* wt, int num_sms);
// api.cu / eval.cu helpers for the surrogate
Plan* kifmm_plan_internal(kifmm_plan_t h);
int kifmm_scatter_weights(Plan& p, const double* I, cudaStream_t st);
// eval.cu
int build_eval_data(Plan& p);
int run_eval(Plan& p, const void* I, void* S, int dtype, double C);

}  // namespace kifmm
