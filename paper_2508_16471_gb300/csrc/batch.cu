// Multi-body batches: the Eq. 24 operator and GMRES over many bodies of
// uneven grids at once.
//
// Every body keeps its own operator (kernel spectrum for its h, voxel map,
// contrast) on a padded size that is a power of two per body.  The solver
// sees one operator (`master`) over all (body, RHS) rows, each row a compact
// vector [3][Nmax] with the batch's largest body size as component stride
// (entries beyond a body's own size stay zero).  Its FP32 application runs the
// five passes over all rows of all bodies that share a padded size in one
// launch per pass (slot descriptors, matvec_fast.cu); the refinement residual
// runs each body's own FP64-accuracy operator on that body's rows.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "farfield.cuh"

namespace vie {

struct BatchBody {
    Operator op;
    std::vector<int> vox_host;
};

struct BatchOps {
    std::vector<BatchBody*> bodies;
    int Rb = 0;             // RHS per body of the current solve / apply
    long long Nmax = 0;     // largest body size (component stride of the rows)
    c32* A = nullptr;       // FP32 work: z-pass output of the slots of one launch
    c32* B = nullptr;       // y-pass output (x pass in place)
    size_t capA = 0, capB = 0;  // elements
    MSlot* d_slots = nullptr;
    int slot_cap = 0;
    std::vector<MSlot> h_slots;
};

}  // namespace vie

struct vie_batch {
    vie::Operator master;
    vie::Solver S;
    vie::BatchOps B;
    int device = 0;
    int n_rhs = 0;
    bool have_solution = false;
};

namespace vie {

static int batch_reserve(Operator& master, BatchOps& bo, size_t needA, size_t needB) {
    if (needA > bo.capA) {
        if (bo.A) dev_free(master, bo.A, sizeof(c32) * bo.capA);
        bo.A = nullptr;
        bo.capA = 0;
        VIE_TRY(dev_alloc(master, (void**)&bo.A, sizeof(c32) * needA));
        bo.capA = needA;
    }
    if (needB > bo.capB) {
        if (bo.B) dev_free(master, bo.B, sizeof(c32) * bo.capB);
        bo.B = nullptr;
        bo.capB = 0;
        VIE_TRY(dev_alloc(master, (void**)&bo.B, sizeof(c32) * needB));
        bo.capB = needB;
    }
    return VIE_OK;
}

// One launch per pass for the listed slots of one padded size.
static int launch_group(Operator& master, BatchOps& bo, const std::vector<int>& rows, int L, const c32* w,
                        long long wr, c32* y, long long yr) {
    const int NL = multi_lines_per_cta(L);
    // the slots' work areas, in chunks that fit the workspace cap (24 GB or 45 % of the free memory)
    size_t fr = 0, tot = 0;
    double limit = 24e9;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess)
        limit = std::max(limit, 0.45 * ((double)fr + sizeof(c32) * (double)(bo.capA + bo.capB)));
    else
        cudaGetLastError();
    size_t i = 0;
    while (i < rows.size()) {
        bo.h_slots.clear();
        long long aoff = 0, boff = 0, zb = 0, yb = 0;
        while (i < rows.size()) {
            const int r = rows[i];
            const Operator& op = bo.bodies[r / bo.Rb]->op;
            const long long sa = 3LL * op.n[0] * op.n[1] * L, sb = 3LL * op.n[0] * L * L;
            if (!bo.h_slots.empty() && sizeof(c32) * (double)(aoff + sa + boff + sb) > limit) break;
            MSlot m;
            m.w = w + r * wr;
            m.y = y + r * yr;
            m.idx = op.idx_map;
            m.chi = op.chi32;
            m.khat = op.khat32;
            m.a_off = aoff;
            m.b_off = boff;
            m.zb0 = zb;
            m.yb0 = yb;
            m.n0 = op.n[0];
            m.n1 = op.n[1];
            m.n2 = op.n[2];
            m.pad = 0;
            bo.h_slots.push_back(m);
            aoff += sa;
            boff += sb;
            zb += (3LL * op.n[0] * op.n[1] + NL - 1) / NL;
            yb += 3LL * op.n[0] * ((L + 15) / 16);  // y-pass column tiles of 16 (AX_TW)
            ++i;
        }
        const int ns = (int)bo.h_slots.size();
        VIE_TRY(batch_reserve(master, bo, (size_t)aoff, (size_t)boff));
        if (ns > bo.slot_cap) {
            if (bo.d_slots) dev_free(master, bo.d_slots, sizeof(MSlot) * bo.slot_cap);
            bo.d_slots = nullptr;
            bo.slot_cap = 0;
            VIE_TRY(dev_alloc(master, (void**)&bo.d_slots, sizeof(MSlot) * std::max(ns, 64)));
            bo.slot_cap = std::max(ns, 64);
        }
        // stream-ordered after the previous launch's kernels; the pageable source is staged before the call returns
        VIE_CUDA(cudaMemcpyAsync(bo.d_slots, bo.h_slots.data(), sizeof(MSlot) * ns, cudaMemcpyHostToDevice,
                                 master.stream));
        const Operator& op0 = bo.bodies[rows[i - 1] / bo.Rb]->op;  // twiddles depend on L only
        VIE_TRY(fast_multi_apply(bo.d_slots, ns, zb, yb, bo.A, bo.B, bo.Nmax, L, op0.H, op0.ax[0].roots32,
                                 op0.ax[1].roots32, op0.ax[2].roots32, master.stream));
    }
    return VIE_OK;
}

int batch_apply(Operator& master, int prec, const void* w, long long wr, void* y, long long yr, int nr) {
    BatchOps& bo = *master.batch;
    const std::vector<int> rows(master.h_list.begin(), master.h_list.begin() + nr);
    if (prec == VIE_PREC_MIXED) {
        // rows of each padded size, in list order (bodies consecutive)
        std::vector<int> sizes;
        for (int r : rows) {
            const int L = bo.bodies[r / bo.Rb]->op.P[0];
            if (std::find(sizes.begin(), sizes.end(), L) == sizes.end()) sizes.push_back(L);
        }
        for (int L : sizes) {
            std::vector<int> g;
            for (int r : rows)
                if (bo.bodies[r / bo.Rb]->op.P[0] == L) g.push_back(r);
            VIE_TRY(launch_group(master, bo, g, L, (const c32*)w, wr, (c32*)y, yr));
        }
        return VIE_OK;
    }
    // FP64 or double-float: each body's own operator on its rows
    size_t i = 0;
    while (i < rows.size()) {
        const int b = rows[i] / bo.Rb;
        std::vector<int> sub;
        while (i < rows.size() && rows[i] / bo.Rb == b) sub.push_back(rows[i++]);
        Operator& op = bo.bodies[b]->op;
        VIE_TRY(op_set_list(op, sub.data(), (int)sub.size()));
        VIE_TRY(op_apply(op, prec, w, wr, y, yr, op.d_list, (int)sub.size()));
    }
    return VIE_OK;
}

static int body_padded(const int n[3]) {
    int need = 1;
    for (int a = 0; a < 3; ++a) need = std::max(need, 2 * n[a] - 1);
    int p = 32;
    while (p < need) p *= 2;
    return p;
}

static void batch_free(vie_batch* bt) {
    if (!bt) return;
    cudaSetDevice(bt->device);
    if (bt->master.stream) cudaStreamSynchronize(bt->master.stream);
    bt->S.release(bt->master);
    for (BatchBody* b : bt->B.bodies) {
        b->op.stream = nullptr;  // the master's stream
        op_free(b->op);
        delete b;
    }
    cudaFree(bt->B.A);
    cudaFree(bt->B.B);
    cudaFree(bt->B.d_slots);
    cudaFree(bt->master.d_list);
    if (bt->master.stream) cudaStreamDestroy(bt->master.stream);
    delete bt;
}

}  // namespace vie

using namespace vie;

extern "C" {

int vie_batch_create(int n_bodies, const vie_grid* grids, const double* const* eps_r, double k0, vie_batch** out) {
    if (!out) return fail(VIE_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_bodies < 1 || n_bodies > 4096 || !grids || !eps_r) return fail(VIE_EINVAL, "bad arguments");
    if (!(k0 > 0) || !std::isfinite(k0)) return fail(VIE_EINVAL, "k0 must be positive and finite");
    for (int b = 0; b < n_bodies; ++b) {
        const vie_grid& g = grids[b];
        for (int a = 0; a < 3; ++a)
            if (g.n[a] < 1 || g.n[a] > 128) return fail(VIE_EINVAL, "batched bodies take 1..128 voxels per axis");
        if (!(g.h > 0) || !std::isfinite(g.h)) return fail(VIE_EINVAL, "voxel size h must be positive and finite");
        if (!eps_r[b]) return fail(VIE_EINVAL, "eps_r is NULL");
        const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
        long long nb = 0;
        for (long long i = 0; i < N; ++i) {
            const double e = eps_r[b][i];
            if (!std::isfinite(e) || e < 1.0) return fail(VIE_EINVAL, "eps_r must be finite and >= 1");
            nb += e > 1.0;
        }
        if (nb == 0) return fail(VIE_EINVAL, "a body is empty (no voxel with eps_r > 1)");
    }
    vie_batch* bt = new vie_batch();
    int st = VIE_OK;
    cudaError_t e = cudaGetDevice(&bt->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bt->master.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) st = cuda_fail(e, "device / stream setup");
    double* deps = nullptr;
    for (int b = 0; b < n_bodies && st == VIE_OK; ++b) {
        BatchBody* bb = new BatchBody();
        bt->B.bodies.push_back(bb);
        Operator& op = bb->op;
        const vie_grid& g = grids[b];
        for (int a = 0; a < 3; ++a) {
            op.n[a] = g.n[a];
            op.origin[a] = g.origin[a];
        }
        op.N = (long long)g.n[0] * g.n[1] * g.n[2];
        op.h = g.h;
        op.k0 = k0;
        op.stream = bt->master.stream;
        const int P = body_padded(op.n);
        for (int a = 0; a < 3; ++a) op.P_fixed[a] = P;
        st = op_init_axes(op);
        if (st == VIE_OK) st = op_build_kernel(op);
        if (st == VIE_OK) {
            e = cudaMalloc(&deps, sizeof(double) * op.N);
            if (e == cudaSuccess) e = cudaMemcpy(deps, eps_r[b], sizeof(double) * op.N, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) st = cuda_fail(e, "eps upload");
        }
        if (st == VIE_OK) st = op_set_body_device(op, deps);
        cudaFree(deps);
        deps = nullptr;
        if (st == VIE_OK) {
            bb->vox_host.resize(op.Nb);
            e = cudaMemcpy(bb->vox_host.data(), op.vox, sizeof(int) * op.Nb, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) st = cuda_fail(e, "voxel list");
        }
        if (st == VIE_OK) {
            bt->B.Nmax = std::max(bt->B.Nmax, op.Nb);
            op.cstride = 0;  // set per call
        }
    }
    if (st != VIE_OK) {
        batch_free(bt);
        return st;
    }
    for (BatchBody* bb : bt->B.bodies) bb->op.cstride = bt->B.Nmax;
    bt->master.Nb = bt->B.Nmax;
    bt->master.batch = &bt->B;
    *out = bt;
    return VIE_OK;
}

void vie_batch_destroy(vie_batch* bt) { batch_free(bt); }

long long vie_batch_stride(const vie_batch* bt) { return bt ? bt->B.Nmax : 0; }

int vie_batch_info(const vie_batch* bt, int body, vie_info* info) {
    if (!bt || !info || body < 0 || body >= (int)bt->B.bodies.size()) return fail(VIE_EINVAL, "bad arguments");
    const Operator& op = bt->B.bodies[body]->op;
    for (int a = 0; a < 3; ++a) {
        info->n[a] = op.n[a];
        info->P[a] = op.P[a];
    }
    info->n_body = op.Nb;
    info->n_rhs = bt->n_rhs;
    info->device = bt->device;
    double bytes = bt->master.bytes;
    for (const BatchBody* b : bt->B.bodies) bytes += b->op.bytes;
    info->device_bytes = bytes;
    return VIE_OK;
}

int vie_batch_apply_device(vie_batch* bt, const void* w_dev, void* y_dev, int n_rhs, int precision) {
    if (!bt || !w_dev || !y_dev || n_rhs < 1) return fail(VIE_EINVAL, "bad arguments");
    if (precision != VIE_PREC_MIXED && precision != VIE_PREC_FP64 && precision != VIE_PREC_F32X2)
        return fail(VIE_EINVAL, "bad precision");
    VIE_CUDA(cudaSetDevice(bt->device));
    const int R = n_rhs * (int)bt->B.bodies.size();
    std::vector<int> list(R);
    for (int r = 0; r < R; ++r) list[r] = r;
    bt->B.Rb = n_rhs;
    VIE_TRY(op_set_list(bt->master, list.data(), R));
    const long long n3 = 3 * bt->B.Nmax;
    return op_apply(bt->master, precision, w_dev, n3, y_dev, n3, bt->master.d_list, R);
}

int vie_batch_solve(vie_batch* bt, const vie_channel* ch, int n_rhs, const vie_solve_opts* opts,
                    vie_solve_stats* stats) {
    if (!bt || !ch) return fail(VIE_EINVAL, "NULL argument");
    const int NB = (int)bt->B.bodies.size();
    if (n_rhs < 1 || (long long)n_rhs * NB > 65535) return fail(VIE_EINVAL, "n_rhs x bodies must be in 1..65535");
    vie_solve_opts o;
    if (opts) o = *opts;
    else vie_default_opts(&o);
    if (!(o.tol > 0) || o.restart < 1 || o.restart > MAX_RESTART || o.max_iter < 1 || !(o.inner_tol > 0) ||
        o.precision != VIE_PREC_MIXED || o.solver != VIE_SOLVER_GMRES || o.precond != 0 || o.use_x0 != 0 ||
        !(o.inner_floor > 0) || !(o.inner_floor <= 1) || !(o.reorth_eta >= 0) || (o.arnoldi != 0 && o.arnoldi != 1))
        return fail(VIE_EINVAL, "batched solves take mixed-precision GMRES from x0 = 0 without a preconditioner");
    for (int r = 0; r < n_rhs; ++r) {
        double kn = 0;
        for (int q = 0; q < 3; ++q) kn += ch[r].khat[q] * ch[r].khat[q];
        const double* p = ch[r].pol;
        const double dr = p[0] * ch[r].khat[0] + p[2] * ch[r].khat[1] + p[4] * ch[r].khat[2];
        const double di = p[1] * ch[r].khat[0] + p[3] * ch[r].khat[1] + p[5] * ch[r].khat[2];
        if (!std::isfinite(kn) || std::fabs(kn - 1.0) > 1e-9) return fail(VIE_EINVAL, "khat must be a unit vector");
        if (std::sqrt(dr * dr + di * di) > 1e-10) return fail(VIE_EINVAL, "polarisation must be transverse");
    }
    VIE_CUDA(cudaSetDevice(bt->device));
    auto t0 = std::chrono::steady_clock::now();
    const int R = n_rhs * NB;
    bt->B.Rb = n_rhs;
    bt->have_solution = false;
    VIE_TRY(bt->S.alloc(bt->master, R, o.restart, o.precision));
    Solver& S = bt->S;
    // entries beyond a body's own size stay zero in every vector of the solve
    VIE_CUDA(cudaMemsetAsync(S.x, 0, sizeof(c64) * S.n3 * R, bt->master.stream));
    VIE_CUDA(cudaMemsetAsync(S.b, 0, sizeof(c64) * S.n3 * R, bt->master.stream));
    VIE_CUDA(cudaMemsetAsync(S.res, 0, sizeof(c64) * S.n3 * R, bt->master.stream));
    VIE_CUDA(cudaMemsetAsync(S.V, 0, sizeof(c32) * S.n3 * R * (size_t)(S.m + 1), bt->master.stream));
    for (int b = 0; b < NB; ++b)
        VIE_TRY(build_rhs_rows(bt->B.bodies[b]->op, S.b + (long long)b * n_rhs * S.n3, S.n3,
                               S.chans + 9LL * b * n_rhs, ch, n_rhs));
    SolveResult res;
    S.pc = nullptr;
    S.bpc = nullptr;
    int st = solver_run(bt->master, S, o, res);
    VIE_CUDA(cudaStreamSynchronize(bt->master.stream));
    auto t1 = std::chrono::steady_clock::now();
    if (st != VIE_OK) return st;
    bt->n_rhs = n_rhs;
    bt->have_solution = true;
    if (stats) {
        stats->n_rhs = R;
        stats->converged = res.converged;
        stats->iters_max = res.iters_max;
        stats->outer_max = res.outer_max;
        stats->matvecs32 = res.matvecs32;
        stats->matvecs64 = res.matvecs64;
        stats->relres_max = res.relres_max;
        stats->seconds = std::chrono::duration<double>(t1 - t0).count();
        if (stats->iters)
            for (int r = 0; r < R; ++r) stats->iters[r] = res.iters[r];
        if (stats->relres)
            for (int r = 0; r < R; ++r) stats->relres[r] = res.relres[r];
    }
    if (res.converged < R)
        return fail(VIE_ENOCONV, "solve stopped before reaching tol; largest FP64 residual " +
                                     std::to_string(res.relres_max));
    return VIE_OK;
}

int vie_batch_get_current(vie_batch* bt, int body, int rhs, double* out) {
    if (!bt || !out) return fail(VIE_EINVAL, "NULL argument");
    if (!bt->have_solution) return fail(VIE_ESTATE, "no solution stored");
    if (body < 0 || body >= (int)bt->B.bodies.size() || rhs < 0 || rhs >= bt->n_rhs)
        return fail(VIE_EINVAL, "body or rhs index out of range");
    const BatchBody& bb = *bt->B.bodies[body];
    const long long Nb = bb.op.Nb, N = bb.op.N, cst = bt->B.Nmax;
    std::vector<c64> buf(3 * cst);
    VIE_CUDA(cudaSetDevice(bt->device));
    VIE_CUDA(cudaMemcpy(buf.data(), bt->S.x + ((long long)body * bt->n_rhs + rhs) * bt->S.n3, sizeof(c64) * 3 * cst,
                        cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(double) * 6 * N);
    for (int c = 0; c < 3; ++c)
        for (long long v = 0; v < Nb; ++v) {
            const long long o = (c * N + bb.vox_host[v]) * 2;
            out[o] = buf[c * cst + v].x;
            out[o + 1] = buf[c * cst + v].y;
        }
    return VIE_OK;
}

int vie_batch_farfield_dirs(vie_batch* bt, int body, const double* dirs, int D, int basis, double* out) {
    if (!bt || !dirs || !out || D < 1) return fail(VIE_EINVAL, "bad arguments");
    if (basis < 0 || basis > 2) return fail(VIE_EINVAL, "basis must be 0, 1 or 2");
    if (!bt->have_solution) return fail(VIE_ESTATE, "no solution stored");
    if (body < 0 || body >= (int)bt->B.bodies.size()) return fail(VIE_EINVAL, "body index out of range");
    VIE_CUDA(cudaSetDevice(bt->device));
    Operator& op = bt->B.bodies[body]->op;
    double* dd = nullptr;
    c64* dout = nullptr;
    VIE_CUDA(cudaMalloc(&dd, sizeof(double) * 3 * D));
    cudaError_t e = cudaMalloc(&dout, sizeof(c64) * 3 * (size_t)D * bt->n_rhs);
    int st = VIE_OK;
    if (e == cudaSuccess) e = cudaMemcpy(dd, dirs, sizeof(double) * 3 * D, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = cuda_fail(e, "far-field buffers");
    if (st == VIE_OK)
        st = farfield_dirs(op, bt->S.x + (long long)body * bt->n_rhs * bt->S.n3, bt->S.n3, bt->n_rhs, dd, D, basis,
                           dout);
    if (st == VIE_OK) {
        e = cudaMemcpy(out, dout, sizeof(c64) * 3 * (size_t)D * bt->n_rhs, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "far-field copy");
    }
    cudaFree(dd);
    cudaFree(dout);
    return st;
}

}  // extern "C"
