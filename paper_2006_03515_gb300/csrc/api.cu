// The C-ABI (include/kifmm.h): argument checks, plan lifetime, evaluation entry points.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.cuh"

namespace kifmm {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

// Plans are identified by a counter that is never reused, not by their heap address (a new
// plan may be created at a destroyed plan's address).
static std::atomic<uint64_t> g_next_uid{1};

// Reads the plan's device error word after its stream has drained: a bounded wait that gave
// up (tensor-core pipelines) leaves a nonzero code there. The word is cleared, so that each
// such event is reported once. Synchronises the plan's stream.
static int take_device_error(Plan& p, const char* who) {
    if (!p.err.p) return KIFMM_OK;
    int e = 0;
    KF_CUDA(cudaStreamSynchronize(p.stream));
    KF_CUDA(cudaMemcpy(&e, p.err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (e == 0) return KIFMM_OK;
    const int zero = 0;
    KF_CUDA(cudaMemcpy(p.err.p, &zero, sizeof(int), cudaMemcpyHostToDevice));
    set_error(std::string(who) + ": a bounded device wait ran out (code " + std::to_string(e) +
              "); the result of the evaluation is not valid");
    return KIFMM_ERR_TIMEOUT;
}

__global__ void gather_sorted_points(const double* pts, const int32_t* perm, int64_t n, double* out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t i = perm[k];
    out[3 * k] = pts[3 * i];
    out[3 * k + 1] = pts[3 * i + 1];
    out[3 * k + 2] = pts[3 * i + 2];
}

static void free_plan(Plan* p) {
    if (!p) return;
    // a batch may have run this plan's work on another plan's lanes: wait for the device
    cudaDeviceSynchronize();
    Tree& t = p->tree;
    for (DevBuf* b : {&t.keys, &t.perm, &t.level, &t.anchor, &t.mcode, &t.parent, &t.child, &t.pstart,
                      &t.pend, &t.leaf, &t.centre})
        dev_free(*b);
    for (auto& L : p->lists) {
        dev_free(L.off);
        dev_free(L.items);
    }
    dev_free(p->vtab);
    for (auto& o : p->ops)
        for (DevBuf* b : {&o.G1, &o.Vb, &o.Ub, &o.Vt, &o.T, &o.Mc, &o.Lo, &o.T32, &o.Ub32, &o.Vb32, &o.Vt32, &o.Lo32, &o.Mc32, &o.ozG1, &o.ozEr,
                          &o.Thi, &o.Tlo, &o.Lhi, &o.Llo, &o.Mhi, &o.Mlo})
            dev_free(*b);
    for (DevBuf* b : {&p->surf, &p->ctab, &p->ctab32, &p->cheb_A, &p->pts, &p->loc32, &p->w, &p->sigma, &p->leaf_of, &p->leaves, &p->p2m_boxes,
                      &p->q, &p->Isort, &p->chk, &p->chkx, &p->cu, &p->cu32, &p->chi, &p->clo, &p->cexp, &p->ozBox, &p->ozEb, &p->dd, &p->phid, &p->phiu,
                      &p->far, &p->wleaves, &p->host_I, &p->host_S, &p->err,
                      &p->tc_tiles, &p->tc_boxes, &p->tc_slots, &p->ptab, &p->l2l_slots, &p->m2m_tiles, &p->m2m_slots, &p->stage32, &p->m2m_hi, &p->m2m_lo, &p->apply_part, &p->nf_utab, &p->nf_Thi, &p->nf_Tlo, &p->nf_tiles,
                      &p->nf_slots, &p->nf_boxes, &p->nf_qhi, &p->nf_qlo, &p->nf_qexp, &p->nf_near, &p->lat_P, &p->lat_Q, &p->lat_Thi, &p->lat_Tlo, &p->lat_iota, &p->lat_slots, &p->lat_fst, &p->lat_Mimg, &p->lat_Mer, &p->nf_ref})
        dev_free(*b);
    for (auto& L : p->lv) {
        for (DevBuf* b : {&L.all, &L.leafs, &L.nonleaf, &L.m2l_tiles, &L.m2l_slots, &L.m2l_slot_off, &L.xboxes,
                          &L.m2l_slots128, &L.m2l_boxes, &L.parents, &L.par_kids, &L.upb,
                          &L.l2l_src, &L.l2l_dst, &L.l2l_off})
            dev_free(*b);
        for (int o = 0; o < 8; ++o) {
            dev_free(L.m2m_src[o]);
            dev_free(L.m2m_dst[o]);
        }
    }
    for (auto& e : p->ev)
        if (e) cudaEventDestroy(e);
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    for (auto s : p->lanes) cudaStreamDestroy(s);
    for (auto e : p->lane_ev) cudaEventDestroy(e);
    if (p->near_st) cudaStreamDestroy(p->near_st);
    for (auto e : p->near_ev)
        if (e) cudaEventDestroy(e);
    for (auto e : p->near_tev)
        if (e) cudaEventDestroy(e);
    delete p;
}

}  // namespace kifmm

using namespace kifmm;

struct kifmm_plan_s {
    Plan* p;
};

namespace kifmm {
Plan* kifmm_plan_internal(kifmm_plan_t h) { return h ? h->p : nullptr; }
}  // namespace kifmm

extern "C" {

void kifmm_default_opts(kifmm_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = KIFMM_FP64;
    o->self_mode = KIFMM_SELF_CELL_EXACT;
    o->pinv_eps = 1e-5;
    o->has_root = 0;
    o->stream = nullptr;
    o->radii[0] = kRInner;
    o->radii[1] = kROuter;
}

const char* kifmm_last_error(void) { return g_last_error.c_str(); }

int kifmm_plan(kifmm_plan_t* out, const double* points, int64_t n, const double* cell_h, double uniform_h,
               int leaf_size, int surface_order, double a, double b, const kifmm_opts* opts_in) {
    set_error("");
    if (!out) {
        set_error("kifmm_plan: out is NULL");
        return KIFMM_ERR_ARG;
    }
    *out = nullptr;
    kifmm_opts o;
    if (opts_in) o = *opts_in;
    else kifmm_default_opts(&o);
    if (!points || n < 1 || n >= (int64_t)1 << 31) {
        set_error("kifmm_plan: need points != NULL and 1 <= n < 2^31");
        return KIFMM_ERR_ARG;
    }
    const bool rect = o.cell_dims[0] != 0.0 || o.cell_dims[1] != 0.0 || o.cell_dims[2] != 0.0;
    if (rect) {
        for (int k = 0; k < 3; ++k)
            if (!(o.cell_dims[k] > 0.0 && std::isfinite(o.cell_dims[k]))) {
                set_error("kifmm_plan: cell_dims must be three finite values > 0 (or all 0)");
                return KIFMM_ERR_ARG;
            }
        if (cell_h) {
            set_error("kifmm_plan: cell_dims and per-point cell_h exclude each other");
            return KIFMM_ERR_ARG;
        }
        uniform_h = std::cbrt(o.cell_dims[0] * o.cell_dims[1] * o.cell_dims[2]);
    } else if (!cell_h && !(uniform_h > 0.0 && std::isfinite(uniform_h))) {
        set_error("kifmm_plan: uniform_h must be finite and > 0 when cell_h is NULL");
        return KIFMM_ERR_ARG;
    }
    if (o.repr != KIFMM_REPR_SURFACE && o.repr != KIFMM_REPR_CHEB) {
        set_error("kifmm_plan: unknown repr");
        return KIFMM_ERR_ARG;
    }
    if (o.repr == KIFMM_REPR_SURFACE && (leaf_size < 1 || surface_order < 3 || surface_order > 12)) {
        set_error("kifmm_plan: need leaf_size >= 1 and 3 <= surface_order <= 12");
        return KIFMM_ERR_ARG;
    }
    if (o.repr == KIFMM_REPR_CHEB && (leaf_size < 1 || surface_order < 2 || surface_order > 10)) {
        set_error("kifmm_plan: need leaf_size >= 1 and 2 <= p <= 10 for the Chebyshev representation");
        return KIFMM_ERR_ARG;
    }
    if (!(a > 0.0) || !(b > a) || !std::isfinite(b)) {
        set_error("kifmm_plan: need 0 < a < b (finite)");
        return KIFMM_ERR_ARG;
    }
    if (o.precision != KIFMM_FP64 && o.precision != KIFMM_MIXED) {
        set_error("kifmm_plan: unknown precision");
        return KIFMM_ERR_ARG;
    }
    if (o.self_mode != KIFMM_SELF_CELL_EXACT && o.self_mode != KIFMM_SELF_PAPER_GL2) {
        set_error("kifmm_plan: unknown self_mode");
        return KIFMM_ERR_ARG;
    }
    if (o.kernel < KIFMM_KERNEL_ZHELEZNYAK || o.kernel > KIFMM_KERNEL_THREEGROUP) {
        set_error("kifmm_plan: unknown kernel");
        return KIFMM_ERR_ARG;
    }
    if (o.kernel != KIFMM_KERNEL_ZHELEZNYAK && o.precision != KIFMM_FP64) {
        set_error("kifmm_plan: the comparison kernels run in the FP64 form");
        return KIFMM_ERR_ARG;
    }
    if (!(o.pinv_eps > 0.0 && o.pinv_eps < 1.0)) {
        set_error("kifmm_plan: pinv_eps must lie in (0, 1)");
        return KIFMM_ERR_ARG;
    }
    if (o.radii[0] == 0.0 && o.radii[1] == 0.0) {
        o.radii[0] = kRInner;
        o.radii[1] = kROuter;
    }
    if (!(o.radii[0] > 1.0 && o.radii[1] > o.radii[0] && o.radii[1] < 3.0)) {
        set_error("kifmm_plan: need 1 < radii[0] < radii[1] < 3");
        return KIFMM_ERR_ARG;
    }
    if (o.has_root && !(o.root[3] > 0.0 && std::isfinite(o.root[3]))) {
        set_error("kifmm_plan: root side must be finite and > 0");
        return KIFMM_ERR_ARG;
    }
    AllocFaultScope fault_scope;
    Plan* p = new (std::nothrow) Plan();
    if (!p) {
        set_error("kifmm_plan: host allocation failed");
        return KIFMM_ERR_OOM;
    }
    p->precision = o.precision;
    p->self_mode = o.self_mode;
    p->kind = o.kernel;
    p->pinv_eps = o.pinv_eps;
    p->r_in = o.radii[0];
    p->r_out = o.radii[1];
    p->stream = (cudaStream_t)o.stream;
    p->a = a;
    p->b = b;
    p->m0 = surface_order;
    p->cheb = o.repr == KIFMM_REPR_CHEB;
    p->S = p->cheb ? surface_order * surface_order * surface_order
                   : surface_order * surface_order * surface_order -
                         (surface_order - 2) * (surface_order - 2) * (surface_order - 2);
    p->Sp = (p->S + 31) / 32 * 32;
    p->leaf_size = leaf_size;
    p->tree.n = n;
    p->n_real = n;
    p->rect = rect && !(o.cell_dims[0] == o.cell_dims[1] && o.cell_dims[1] == o.cell_dims[2]);
    if (rect && !p->rect) uniform_h = o.cell_dims[0];   // equal sides: a cube
    for (int k = 0; k < 3; ++k) p->cell_dims[k] = p->rect ? o.cell_dims[k] : 0.0;
    auto fail = [&](int rc) {
        std::string msg = g_last_error;
        free_plan(p);
        cudaGetLastError();
        g_last_error = msg;
        return rc;
    };
    DevBuf padded;   // the caller's points and the padding cells (plan time only)
    int nc = 1;
    while ((nc + 1) * (nc + 1) * (nc + 1) <= leaf_size) ++nc;
    if (o.pad_lattice && !cell_h && !rect && !o.has_root && nc >= 2 && nc * nc * nc == leaf_size) {
        int64_t nt = n;
        double root[4];
        int prc = pad_to_lattice(p->stream, points, n, uniform_h, nc, padded, &nt, root);
        if (prc) {
            dev_free(padded);
            return fail(prc);
        }
        if (nt > n) {
            points = static_cast<const double*>(padded.p);
            p->tree.n = n = nt;
        }
        if (root[3] > 0.0) {   // a box grid: the root on its leaf lattice (padded or not)
            o.has_root = 1;
            for (int k = 0; k < 4; ++k) o.root[k] = root[k];
        }
    }
    int rc = build_tree(*p, points, cell_h, uniform_h, o);
    if (!rc) rc = dev_alloc(p->pts, n * 3 * sizeof(double));
    if (rc) {
        dev_free(padded);
        return fail(rc);
    }
    gather_sorted_points<<<(unsigned)((n + 255) / 256), 256, 0, p->stream>>>(points, ptr<int32_t>(p->tree.perm), n,
                                                                           ptr<double>(p->pts));
    if (cudaGetLastError() != cudaSuccess) {
        dev_free(padded);
        set_error("kifmm_plan: launch failed");
        return fail(KIFMM_ERR_CUDA);
    }
    if (padded.p) {   // the plan keeps its own sorted copy
        if (cudaStreamSynchronize(p->stream) != cudaSuccess) {
            dev_free(padded);
            return fail(KIFMM_ERR_CUDA);
        }
        dev_free(padded);
    }
    rc = build_lists(*p);
    if (rc) return fail(rc);
    rc = build_operators(*p);
    if (rc) return fail(rc);
    rc = build_self_terms(*p, cell_h, uniform_h);
    if (rc) return fail(rc);
    rc = dev_alloc(p->err, 16);
    if (rc) return fail(rc);
    if (cudaMemsetAsync(p->err.p, 0, 16, p->stream) != cudaSuccess) return fail(KIFMM_ERR_CUDA);
    {   // KIFMM_INJECT_DEVICE_ERROR=code: the word starts at that code, as if a bounded wait of
        // the plan had given up (tests of the status reporting; no device wait is disturbed)
        const char* inj = std::getenv("KIFMM_INJECT_DEVICE_ERROR");
        const int code = inj ? std::atoi(inj) : 0;
        if (code != 0 &&
            cudaMemcpyAsync(p->err.p, &code, sizeof(int), cudaMemcpyHostToDevice, p->stream) != cudaSuccess)
            return fail(KIFMM_ERR_CUDA);
        if (code != 0 && cudaStreamSynchronize(p->stream) != cudaSuccess) return fail(KIFMM_ERR_CUDA);
    }
    p->uid = g_next_uid.fetch_add(1);
    p->uniform_h = (cell_h || p->rect) ? 0.0 : uniform_h;
    rc = build_eval_data(*p);
    if (rc) return fail(rc);
    rc = dev_alloc(p->host_I, p->n_real * 8);
    if (rc) return fail(rc);
    rc = dev_alloc(p->host_S, p->n_real * 8);
    if (rc) return fail(rc);
    const char* tm = std::getenv("KIFMM_TIMING");
    if (tm && tm[0] == '1') {
        p->timing = true;
        for (auto& e : p->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return fail(KIFMM_ERR_CUDA);
        if (p->near_st)
            for (auto& e : p->near_tev)
                if (cudaEventCreate(&e) != cudaSuccess) return fail(KIFMM_ERR_CUDA);
    }
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) {
        set_error(std::string("kifmm_plan: ") + cudaGetErrorString(cudaGetLastError()));
        return fail(KIFMM_ERR_CUDA);
    }
    kifmm_plan_s* h = new (std::nothrow) kifmm_plan_s{p};
    if (!h) return fail(KIFMM_ERR_OOM);
    *out = h;
    return KIFMM_OK;
}

int kifmm_eval(kifmm_plan_t h, const void* I, void* S, int dtype, double C) {
    if (!h || !h->p || !I || !S || (dtype != KIFMM_F32 && dtype != KIFMM_F64) || !std::isfinite(C)) {
        set_error("kifmm_eval: invalid argument");
        return KIFMM_ERR_ARG;
    }
    Plan& p = *h->p;
    int rc = run_eval(p, I, S, dtype, C);
    if (rc) return rc;
    if (p.timing) {
        cudaEventSynchronize(p.ev[7]);
        for (int k = 0; k < 7; ++k) cudaEventElapsedTime(&p.phase_ms[k], p.ev[k], p.ev[k + 1]);
        p.n_phases = 7;
        if (p.near_forked && p.near_tev[1]) {   // the near sums on their own stream, beside the far field
            cudaEventElapsedTime(&p.phase_ms[7], p.near_tev[0], p.near_tev[1]);
            p.n_phases = 8;
        }
    }
    return KIFMM_OK;
}

int kifmm_eval_host(kifmm_plan_t h, const void* I_host, void* S_host, int dtype, double C) {
    if (!h || !h->p || !I_host || !S_host || (dtype != KIFMM_F32 && dtype != KIFMM_F64)) {
        set_error("kifmm_eval_host: invalid argument");
        return KIFMM_ERR_ARG;
    }
    Plan& p = *h->p;
    size_t bytes = (size_t)p.n_real * (dtype == KIFMM_F64 ? 8 : 4);
    KF_CUDA(cudaMemcpyAsync(p.host_I.p, I_host, bytes, cudaMemcpyHostToDevice, p.stream));
    KF_TRY(kifmm_eval(h, p.host_I.p, p.host_S.p, dtype, C));
    KF_CUDA(cudaMemcpyAsync(S_host, p.host_S.p, bytes, cudaMemcpyDeviceToHost, p.stream));
    KF_CUDA(cudaStreamSynchronize(p.stream));
    return take_device_error(p, "kifmm_eval_host");
}

int kifmm_check(kifmm_plan_t h) {
    if (!h || !h->p) {
        set_error("kifmm_check: invalid argument");
        return KIFMM_ERR_ARG;
    }
    return take_device_error(*h->p, "kifmm_check");
}

// Lane of each batch entry: distinct plans, largest first, each onto the lane with the
// fewest points so far; entries repeating a plan take that plan's lane.
static std::vector<int> assign_lanes(kifmm_plan_t* plans, int count, int lanes) {
    std::vector<int> lane(count, -1), order;
    for (int k = 0; k < count; ++k) {
        bool first = true;
        for (int j = 0; j < k && first; ++j) first = plans[j] != plans[k];
        if (first) order.push_back(k);
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return plans[x]->p->tree.n > plans[y]->p->tree.n; });
    std::vector<int64_t> load(lanes, 0);
    for (int k : order) {
        int best = 0;
        for (int j = 1; j < lanes; ++j)
            if (load[j] < load[best]) best = j;
        load[best] += plans[k]->p->tree.n;
        for (int j = 0; j < count; ++j)
            if (plans[j] == plans[k]) lane[j] = best;
    }
    return lane;
}

int kifmm_eval_batch(kifmm_plan_t* plans, const void* const* I, void* const* S, int count, int dtype,
                     const double* C, int capture, int lanes) {
    if (!plans || !I || !S || count < 1 || lanes < 1 || lanes > KIFMM_MAX_LANES) {
        set_error("kifmm_eval_batch: invalid argument");
        return KIFMM_ERR_ARG;
    }
    for (int k = 0; k < count; ++k)
        if (!plans[k] || !plans[k]->p) {
            set_error("kifmm_eval_batch: NULL plan");
            return KIFMM_ERR_ARG;
        }
    Plan& p0 = *plans[0]->p;
    cudaStream_t st = p0.stream;
    std::vector<int> lane_of = assign_lanes(plans, count, lanes);
    int used = 0;
    for (int l : lane_of) used = std::max(used, l + 1);
    if (used > 1) {
        while ((int)p0.lanes.size() < used) {
            cudaStream_t s;
            KF_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            p0.lanes.push_back(s);
        }
        while ((int)p0.lane_ev.size() < used + 1) {
            cudaEvent_t e;
            KF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            p0.lane_ev.push_back(e);
        }
    }
    // the captured graph holds every argument of the batch: plans (by id), buffers and the
    // per-field scale C (a kernel argument), so any change of them re-captures
    std::vector<uint64_t> key;
    key.reserve(4 * count + 3);
    key.push_back((uint64_t)count);
    key.push_back((uint64_t)dtype);
    key.push_back((uint64_t)used);
    for (int k = 0; k < count; ++k) {
        const double ck = C ? C[k] : 1.0;
        uint64_t cbits;
        std::memcpy(&cbits, &ck, sizeof(cbits));
        key.push_back(plans[k]->p->uid);
        key.push_back((uint64_t)(uintptr_t)I[k]);
        key.push_back((uint64_t)(uintptr_t)S[k]);
        key.push_back(cbits);
    }
    auto run_one = [&](int k, cudaStream_t s) -> int {
        Plan& pk = *plans[k]->p;
        cudaStream_t saved = pk.stream;
        bool saved_t = pk.timing;
        pk.stream = s;
        pk.timing = false;
        int rc = run_eval(pk, I[k], S[k], dtype, C ? C[k] : 1.0);
        pk.stream = saved;
        pk.timing = saved_t;
        return rc;
    };
    auto launch_all = [&]() -> int {
        if (used <= 1) {
            for (int k = 0; k < count; ++k) KF_TRY(run_one(k, st));
            return KIFMM_OK;
        }
        // fork: every lane waits for the work already ordered on plan[0]'s stream
        KF_CUDA(cudaEventRecord(p0.lane_ev[0], st));
        for (int j = 0; j < used; ++j) KF_CUDA(cudaStreamWaitEvent(p0.lanes[j], p0.lane_ev[0], 0));
        int rc = KIFMM_OK;
        for (int k = 0; k < count && rc == KIFMM_OK; ++k) rc = run_one(k, p0.lanes[lane_of[k]]);
        // join every forked lane, also after a failure (a capture needs its forks joined)
        for (int j = 0; j < used; ++j) {
            cudaError_t e = cudaEventRecord(p0.lane_ev[1 + j], p0.lanes[j]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p0.lane_ev[1 + j], 0);
            if (e != cudaSuccess && rc == KIFMM_OK) {
                set_error(std::string("kifmm_eval_batch: lane join: ") + cudaGetErrorString(e));
                rc = KIFMM_ERR_CUDA;
            }
        }
        return rc;
    };
    if (!capture) return launch_all();
    if (p0.graph_exec && p0.graph_key == key) {
        KF_CUDA(cudaGraphLaunch(p0.graph_exec, st));
        return KIFMM_OK;
    }
    if (!st) {
        set_error("kifmm_eval_batch: graph capture needs a non-default stream in plan[0]");
        return KIFMM_ERR_ARG;
    }
    if (p0.graph_exec) {
        cudaGraphExecDestroy(p0.graph_exec);
        p0.graph_exec = nullptr;
    }
    cudaGraph_t g;
    KF_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = launch_all();
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc) {
        if (e == cudaSuccess) cudaGraphDestroy(g);
        return rc;
    }
    KF_CUDA(e);
    cudaError_t ei = cudaGraphInstantiate(&p0.graph_exec, g, 0);
    cudaGraphDestroy(g);
    KF_CUDA(ei);
    p0.graph_key = key;
    KF_CUDA(cudaGraphLaunch(p0.graph_exec, st));
    return KIFMM_OK;
}

__global__ void k_fill_ones(double* x, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = 1.0;
}

int kifmm_autotune(const double* points, int64_t n, const double* cell_h, double uniform_h, const int* cand,
                   int ncand, int surface_order, double a, double b, const kifmm_opts* opts_in, int reps,
                   int* best_leaf, float* ms_out) {
    if (!cand || ncand < 1 || !best_leaf || reps < 1) {
        set_error("kifmm_autotune: need candidates, ncand >= 1, reps >= 1 and best_leaf");
        return KIFMM_ERR_ARG;
    }
    kifmm_opts o;
    if (opts_in) o = *opts_in;
    else kifmm_default_opts(&o);
    cudaStream_t st = (cudaStream_t)o.stream;
    DevBuf I, S;
    KF_TRY(dev_alloc(I, (size_t)std::max<int64_t>(n, 1) * 8));
    int rc = dev_alloc(S, (size_t)std::max<int64_t>(n, 1) * 8);
    if (rc) { dev_free(I); return rc; }
    k_fill_ones<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ptr<double>(I), n);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = 3.0e38f;
    *best_leaf = -1;
    rc = KIFMM_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = KIFMM_ERR_CUDA;
    for (int k = 0; k < ncand && rc == KIFMM_OK; ++k) {
        kifmm_plan_t p = nullptr;
        rc = kifmm_plan(&p, points, n, cell_h, uniform_h, cand[k], surface_order, a, b, &o);
        if (rc) break;
        rc = kifmm_eval(p, I.p, S.p, KIFMM_F64, 1.0);
        float ms = 0.f;
        if (!rc) {
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps && !rc; ++r) rc = kifmm_eval(p, I.p, S.p, KIFMM_F64, 1.0);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                rc = rc ? rc : KIFMM_ERR_CUDA;
            ms /= reps;
        }
        kifmm_destroy(p);
        if (rc) break;
        if (ms_out) ms_out[k] = ms;
        if (ms < best) {
            best = ms;
            *best_leaf = cand[k];
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(I);
    dev_free(S);
    return rc;
}

int kifmm_model_constants(double p, double p_o2, double p_q, double xi_oa, double* a, double* b, double* C) {
    for (double v : {p, p_o2, p_q, xi_oa})
        if (!(v > 0.0) || !std::isfinite(v)) {
            set_error("kifmm_model_constants: pressures and xi (omega/alpha) must be finite and > 0");
            return KIFMM_ERR_ARG;
        }
    // Sec. 2.1: chi_min = 0.035, chi_max = 2 /(cm Torr); Eq. (Ifun): C = xi (omega/alpha) p_q / (p + p_q)
    if (a) *a = 0.035 * p_o2;
    if (b) *b = 2.0 * p_o2;
    if (C) *C = xi_oa * p_q / (p + p_q);
    return KIFMM_OK;
}

void kifmm_destroy(kifmm_plan_t h) {
    if (!h) return;
    free_plan(h->p);
    delete h;
}

int kifmm_get_info(kifmm_plan_t h, kifmm_info* info) {
    if (!h || !h->p || !info) {
        set_error("kifmm_get_info: invalid argument");
        return KIFMM_ERR_ARG;
    }
    Plan& p = *h->p;
    info->n_points = p.tree.n;
    info->n_padding = p.tree.n - p.n_real;
    info->n_boxes = p.tree.nboxes;
    info->n_levels = p.tree.nlevels;
    info->surface_points = p.S;
    info->n_leaves = p.nleaves;
    for (int k = 0; k < 4; ++k) info->list_len[k] = p.lists[k].len;
    for (int k = 0; k < 3; ++k) info->origin[k] = p.tree.origin[k];
    info->side = p.tree.side;
    int rmin = p.S;
    for (int l = 2; l < p.tree.nlevels; ++l) rmin = std::min(rmin, p.ops[l].rank);
    info->pinv_rank_min = rmin;
    info->eval_launches = p.eval_launches;
    info->m2l_tensor = p.m2l_tensor ? 1 : 0;
    info->near_tensor = p.near_tc ? 1 : 0;
    info->lattice_far = p.lat_far ? 1 : 0;
    {   // the same conditions as the evaluation's dispatch of M2M, L2L and the upward solves
        const bool mixed = p.precision == KIFMM_MIXED;
        int64_t nm = 0, nl2 = 0, nup = 0;
        for (int l = 2; l < p.tree.nlevels; ++l) {
            if (p.lv[l].n_par > 0 && mixed && !p.cheb && p.m2m_tc && p.m2m_count[l] >= p.tc_min_tiles) ++nm;
            if (l >= 3 && p.lv[l - 1].l2l_max > 0 && mixed && !p.cheb && p.l2l_tc && p.tc_count[l] >= p.tc_min_tiles)
                ++nl2;
            if (!p.cheb && ((p.lat_up && l == p.nf_level) || (p.oz && p.lv[l].n_up > p.oz_min))) ++nup;
        }
        info->m2m_tensor_levels = nm;
        info->l2l_tensor_levels = nl2;
        info->upward_tensor_levels = nup;
    }
    info->m2l_flops = p.m2l_flops;
    {
        double up = 0;
        // FP64 pseudo-inverse applications c = Sigma^+ U^T chk, one per leaf and per parent
        // (none in the Chebyshev representation)
        if (!p.cheb)   // (the leaves of a lattice plan: 2 r npl each, from their weights)
            for (int l = 2; l < p.tree.nlevels; ++l)
                up += 2.0 * p.ops[l].rank * (p.lat_up && l == p.nf_level ? p.nf_R : p.S) * p.lv[l].n_up;
        info->upward_flops = up;
        double mma = 0;
        if (p.oz)
            for (int l = 2; l < p.tree.nlevels; ++l)
                if (p.lv[l].n_up > p.oz_min)
                    mma += pinv_oz_mma_flops(p.lat_up && l == p.nf_level ? p.nf_R : p.S, p.ops[l].rank, p.lv[l].n_up);
        info->upward_mma_flops = mma;
    }
    info->device_error = 0;
    if (p.err.p) {
        int e = 0;
        KF_CUDA(cudaMemcpyAsync(&e, p.err.p, sizeof(int), cudaMemcpyDeviceToHost, p.stream));
        KF_CUDA(cudaStreamSynchronize(p.stream));
        info->device_error = e;
    }
    info->p2p_pairs = p.p2p_pairs;
    return KIFMM_OK;
}

static int copy_i32_to_i64(const DevBuf& src, int64_t n, int64_t* dst, cudaStream_t st) {
    if (!dst) return KIFMM_OK;
    std::vector<int32_t> tmp(n);
    KF_CUDA(cudaMemcpyAsync(tmp.data(), src.p, n * 4, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < n; ++i) dst[i] = tmp[i];
    return KIFMM_OK;
}

static int copy_raw(const DevBuf& src, size_t bytes, void* dst, cudaStream_t st) {
    if (!dst) return KIFMM_OK;
    KF_CUDA(cudaMemcpyAsync(dst, src.p, bytes, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    return KIFMM_OK;
}

int kifmm_get_tree(kifmm_plan_t h, int64_t* perm, uint64_t* keys, int32_t* level, int32_t* parent,
                   int64_t* pstart, int64_t* pend, int32_t* leaf, int32_t* anchor, int32_t* child) {
    if (!h || !h->p) {
        set_error("kifmm_get_tree: invalid argument");
        return KIFMM_ERR_ARG;
    }
    Plan& p = *h->p;
    Tree& t = p.tree;
    cudaStream_t st = p.stream;
    KF_TRY(copy_i32_to_i64(t.perm, t.n, perm, st));
    KF_TRY(copy_raw(t.keys, t.n * 8, keys, st));
    KF_TRY(copy_raw(t.level, t.nboxes * 4, level, st));
    KF_TRY(copy_raw(t.parent, t.nboxes * 4, parent, st));
    KF_TRY(copy_i32_to_i64(t.pstart, t.nboxes, pstart, st));
    KF_TRY(copy_i32_to_i64(t.pend, t.nboxes, pend, st));
    KF_TRY(copy_raw(t.leaf, t.nboxes * 4, leaf, st));
    KF_TRY(copy_raw(t.anchor, t.nboxes * 12, anchor, st));
    KF_TRY(copy_raw(t.child, t.nboxes * 32, child, st));
    return KIFMM_OK;
}

int kifmm_get_list(kifmm_plan_t h, int which, int64_t* offsets, int32_t* items) {
    if (!h || !h->p || which < 0 || which > 3) {
        set_error("kifmm_get_list: invalid argument");
        return KIFMM_ERR_ARG;
    }
    Plan& p = *h->p;
    KF_TRY(copy_i32_to_i64(p.lists[which].off, p.tree.nboxes + 1, offsets, p.stream));
    KF_TRY(copy_raw(p.lists[which].items, p.lists[which].len * 4, items, p.stream));
    return KIFMM_OK;
}

int kifmm_get_sigma(kifmm_plan_t h, double* sigma) {
    if (!h || !h->p || !sigma) {
        set_error("kifmm_get_sigma: invalid argument");
        return KIFMM_ERR_ARG;
    }
    return copy_raw(h->p->sigma, h->p->tree.n * 8, sigma, h->p->stream);
}

int kifmm_get_upward(kifmm_plan_t h, double* c, int* stride) {
    if (!h || !h->p || !stride) {
        set_error("kifmm_get_upward: invalid argument");
        return KIFMM_ERR_ARG;
    }
    *stride = h->p->R;
    if (!c) return KIFMM_OK;   // stride query
    return copy_raw(h->p->cu, (size_t)h->p->tree.nboxes * h->p->R * 8, c, h->p->stream);
}

int kifmm_get_phase_times(kifmm_plan_t h, float* ms, int cap) {
    if (!h || !h->p || !ms) return 0;
    int n = std::min(cap, h->p->n_phases);
    for (int k = 0; k < n; ++k) ms[k] = h->p->phase_ms[k];
    return n;
}

}  // extern "C"
