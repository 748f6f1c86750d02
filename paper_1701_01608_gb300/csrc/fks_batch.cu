// fks_batch.cu -- uneven batches of space-homogeneous problems behind the fks_batch_* entry points
// of include/fks.h: per-class tables and kernel variants, per-problem descriptors, one persistent
// launch per velocity-grid class on forked streams, and CUDA-graph capture of many steps.
//
// Method: arXiv 1701.01608, Appendix A (fast spectral operator) and Sec. 2.1 (explicit Euler
// collision step), applied to independent space-homogeneous cells.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fks.h"
#include "fks_internal.h"

using namespace fks;

// ------------------------------------------------------------------ uneven batches
//
// A batch holds independent space-homogeneous problems (one cell each) with
// their own n, box L, kernel and Knudsen number.  Problems of one n form one
// class, run by one persistent launch of the batch kernel over per-problem
// descriptors; the classes run concurrently (fork/join on internal streams),
// and fks_batch_run captures many steps of that once in a CUDA graph.
namespace {

struct TableSet {
    int n, ktype;
    double L, Ck;
    void* tables = nullptr;
    void* tables64 = nullptr;   // double-float tables of the escalation tier (FP32 batches)
    double* P = nullptr;   // device, 25 doubles
};

struct BatchClass {
    int n = 0, C = 0, max_clusters = 0;
    CollideVariant var{};
    EscTier esc{};               // FP32 batches: double-float arithmetic over the FP32 state (tables in the TableSets)
    std::vector<int> probs;      // problem indices, in item order
    long first = 0;              // offset of this class in an item array
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

struct ItemSet {
    std::vector<const void*> f;
    std::vector<void*> o;
    std::vector<double> dt;
    BatchItem* d = nullptr;
    BatchItem* d64 = nullptr;    // the same items with the FP64 tables (escalation tier)
};

struct GraphEntry {
    std::vector<const void*> a, b;
    std::vector<double> dt;
    int nsteps = 0;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct fks_batch {
    int nprob = 0, M = 0;
    bool fp64 = false;
    fks_dirs dirs{};
    std::vector<int> n, ktype, tset;
    std::vector<double> L, Ck, kn;
    std::vector<TableSet> tsets;
    std::vector<BatchClass> classes;
    std::vector<ItemSet> items;
    std::vector<GraphEntry> graphs;
    cudaEvent_t fork = nullptr;
    int* d_flags = nullptr;
    long launches = 0;
    std::string err;
    // precision escalation of FP32 batches (as for contexts): problems whose error bound exceeds
    // esc_tol are listed per class and recomputed in FP64 arithmetic
    double esc_tol = 0.0;
    int* esc_lists = nullptr;    // [nprob], class k at its item offset
    int* esc_counts = nullptr;   // [classes]
};

static fks_status bfail(fks_batch* b, fks_status s, const std::string& m) {
    if (b) b->err = m;
    return s;
}

// (re)build the table sets of class k for its current cluster size
static fks_status batch_build_class_tables(fks_batch* b, BatchClass& cl) {
    for (size_t t = 0; t < b->tsets.size(); ++t) {
        TableSet& ts = b->tsets[t];
        if (ts.n != cl.n) continue;
        if (ts.tables) cudaFree(ts.tables);
        ts.tables = nullptr;
        std::string err;
        fks_status st = build_tables_raw(ts.n, b->dirs, ts.L, ts.ktype, ts.Ck, cl.C, b->fp64, &ts.tables, &err);
        if (st != FKS_OK) return bfail(b, st, err);
        b->launches += 2;
    }
    return FKS_OK;
}

// escalation tier of an FP32 class: the batch kernel in double-float arithmetic over the FP32
// state, and double-float tables of every table set of the class
static fks_status batch_setup_escalation(fks_batch* b, BatchClass& cl) {
    EscTier& t = cl.esc;
    t.fp64 = true;
    t.dfl = true;
    t.C = default_cluster_size(true, cl.n);
    if (!find_collide_variant_dfloat(cl.n, t.C, &t.var)) return bfail(b, FKS_ERR_UNSUPPORTED, "no escalation kernel");
    cudaError_t e = cudaFuncSetAttribute(t.var.func_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.var.smem);
    if (e != cudaSuccess) return bfail(b, FKS_ERR_CUDA, cudaGetErrorString(e));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = t.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(t.C, 1, 1);
    cfg.blockDim = dim3(t.var.NT, 1, 1);
    cfg.dynamicSmemBytes = t.var.smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaOccupancyMaxActiveClusters(&t.max_clusters, t.var.func_batch, &cfg);
    if (e != cudaSuccess) return bfail(b, FKS_ERR_CUDA, cudaGetErrorString(e));
    if (t.max_clusters <= 0) return bfail(b, FKS_ERR_UNSUPPORTED, "escalation kernel cannot be resident");
    for (TableSet& ts : b->tsets) {
        if (ts.n != cl.n || ts.tables64) continue;
        std::string err;
        const fks_status st = build_tables_raw(ts.n, b->dirs, ts.L, ts.ktype, ts.Ck, t.C, true, &ts.tables64, &err,
                                               false, nullptr, true);
        if (st != FKS_OK) return bfail(b, st, err);
        b->launches += 2;
    }
    return FKS_OK;
}

static fks_status batch_configure_class(fks_batch* b, BatchClass& cl, int C, int radix = 0) {
    CollideVariant v;
    int nclus = 0;
    bool found = false;
    cudaError_t e = query_variant(b->fp64, cl.n, C, &v, &nclus, &found, radix);
    if (e != cudaSuccess) return bfail(b, FKS_ERR_CUDA, cudaGetErrorString(e));
    if (!found) return bfail(b, FKS_ERR_UNSUPPORTED, "no collision kernel for this (precision, n, cluster size)");
    if (nclus <= 0) return bfail(b, FKS_ERR_UNSUPPORTED, "batch kernel cannot be resident on this device");
    cl.var = v;
    cl.C = C;
    cl.max_clusters = nclus;
    return FKS_OK;
}

// device descriptors for one (f, out, dt) assignment, cached per pointer set
static fks_status batch_items(fks_batch* b, const void* const* f, void* const* o, const double* dt, BatchItem** out) {
    for (ItemSet& s : b->items) {
        bool same = true;
        for (int i = 0; i < b->nprob && same; ++i) same = s.f[i] == f[i] && s.o[i] == o[i] && s.dt[i] == dt[i];
        if (same) {
            *out = s.d;
            return FKS_OK;
        }
    }
    std::vector<BatchItem> h(b->nprob);
    for (const BatchClass& cl : b->classes)
        for (size_t j = 0; j < cl.probs.size(); ++j) {
            const int i = cl.probs[j];
            BatchItem& it = h[cl.first + j];
            it.f = f[i];
            it.out = o[i];
            it.tables = b->tsets[b->tset[i]].tables;
            it.P = b->tsets[b->tset[i]].P;
            it.inv_kn = 1.0 / b->kn[i];
            it.dt = dt[i];
            it.L = b->L[i];
            it.pad_ = 0.0;
        }
    ItemSet s;
    s.f.assign(f, f + b->nprob);
    s.o.assign(o, o + b->nprob);
    s.dt.assign(dt, dt + b->nprob);
    if (cudaMalloc(&s.d, sizeof(BatchItem) * b->nprob) != cudaSuccess) return bfail(b, alloc_failure(), "item descriptors");
    if (cudaMemcpy(s.d, h.data(), sizeof(BatchItem) * b->nprob, cudaMemcpyHostToDevice) != cudaSuccess)
        return bfail(b, FKS_ERR_CUDA, "item upload");
    if (!b->fp64) {
        for (const BatchClass& cl : b->classes)
            for (size_t j = 0; j < cl.probs.size(); ++j) h[cl.first + j].tables = b->tsets[b->tset[cl.probs[j]]].tables64;
        if (cudaMalloc(&s.d64, sizeof(BatchItem) * b->nprob) != cudaSuccess) {
            cudaFree(s.d);
            return bfail(b, alloc_failure(), "item descriptors");
        }
        if (cudaMemcpy(s.d64, h.data(), sizeof(BatchItem) * b->nprob, cudaMemcpyHostToDevice) != cudaSuccess)
            return bfail(b, FKS_ERR_CUDA, "item upload");
    }
    b->items.push_back(s);
    *out = s.d;
    return FKS_OK;
}

// the FP64-table copy of an item array (escalation tier)
static BatchItem* batch_items64(const fks_batch* b, const BatchItem* d) {
    for (const ItemSet& s : b->items)
        if (s.d == d) return s.d64;
    return nullptr;
}

// enqueue one collide (mode 0) or Euler step (mode 1) of every problem on s
static cudaError_t batch_kernel(const CollideVariant& var, int C, int max_clusters, const CollideArgs& a,
                                cudaStream_t cs) {
    const long nclus = a.ncells < max_clusters ? a.ncells : max_clusters;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(nclus * C), 1, 1);
    cfg.blockDim = dim3(var.NT, 1, 1);
    cfg.dynamicSmemBytes = var.smem;
    cfg.stream = cs;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CollideArgs arg = a;
    void* args[] = {&arg};
    return cudaLaunchKernelExC(&cfg, var.func_batch, args);
}

static fks_status batch_launch(fks_batch* b, BatchItem* d_items, int mode, cudaStream_t s) {
    const bool fork = b->classes.size() > 1;
    BatchItem* d64 = (!b->fp64 && b->esc_tol > 0.0) ? batch_items64(b, d_items) : nullptr;
    if (d64 && cudaMemsetAsync(b->esc_counts, 0, sizeof(int) * b->classes.size(), s) != cudaSuccess)
        return bfail(b, FKS_ERR_CUDA, "escalation counts");
    if (fork && cudaEventRecord(b->fork, s) != cudaSuccess) return bfail(b, FKS_ERR_CUDA, "fork event");
    for (size_t k = 0; k < b->classes.size(); ++k) {
        BatchClass& cl = b->classes[k];
        cudaStream_t cs = fork ? cl.stream : s;
        if (fork && cudaStreamWaitEvent(cs, b->fork, 0) != cudaSuccess) return bfail(b, FKS_ERR_CUDA, "fork wait");
        CollideArgs a;
        std::memset(&a, 0, sizeof(a));
        a.items = d_items + cl.first;
        a.ncells = (long)cl.probs.size();
        a.nc[0] = a.nc[1] = a.nc[2] = 1;
        a.M = b->M;
        a.L = b->L[cl.probs[0]];
        a.mode = mode;
        a.flags = b->d_flags;
        if (d64) {
            a.esc_list = b->esc_lists + cl.first;
            a.esc_count = b->esc_counts + k;
            a.esc_c2 = kEscFp32 * kEscFp32;
            a.esc_tol2 = b->esc_tol * b->esc_tol;
        }
        cudaError_t e = batch_kernel(cl.var, cl.C, cl.max_clusters, a, cs);
        if (e != cudaSuccess) return bfail(b, FKS_ERR_CUDA, std::string("batch kernel launch: ") + cudaGetErrorString(e));
        b->launches += 1;
        if (d64) {
            // the listed problems again, in FP64 arithmetic (the count is read on the device)
            a.items = d64 + cl.first;
            a.list = b->esc_lists + cl.first;
            a.list_count = b->esc_counts + k;
            a.esc_list = nullptr;
            a.esc_count = nullptr;
            e = batch_kernel(cl.esc.var, cl.esc.C, cl.esc.max_clusters, a, cs);
            if (e != cudaSuccess)
                return bfail(b, FKS_ERR_CUDA, std::string("escalation kernel launch: ") + cudaGetErrorString(e));
            b->launches += 1;
        }
        if (fork) {
            if (cudaEventRecord(cl.done, cs) != cudaSuccess || cudaStreamWaitEvent(s, cl.done, 0) != cudaSuccess)
                return bfail(b, FKS_ERR_CUDA, "join");
        }
    }
    return FKS_OK;
}

extern "C" {

fks_status fks_batch_init(int nprob, const int* n, const double* L, const int* ktype, const double* C,
                          const double* knudsen, const fks_dirs* dirs, int precision, fks_batch** out) {
    if (out) *out = nullptr;
    if (!out || nprob < 1 || !n || !L || !ktype || !C || !knudsen || !dirs) return FKS_ERR_INVALID_ARG;
    if (precision != FKS_FP64 && precision != FKS_FP32) return FKS_ERR_UNSUPPORTED;
    if (dirs->A1 < 1 || dirs->A2 < 1 || dirs->A1 * dirs->A2 > 4096 || (dirs->rule != 0 && dirs->rule != 1))
        return FKS_ERR_INVALID_ARG;
    for (int i = 0; i < nprob; ++i) {
        if (n[i] != 8 && n[i] != 16 && n[i] != 24 && n[i] != 32) return FKS_ERR_UNSUPPORTED;
        if (ktype[i] == FKS_BGK || ktype[i] == FKS_VHS) return FKS_ERR_UNSUPPORTED;
        if (!(L[i] > 0.0) || !std::isfinite(L[i]) || (ktype[i] != 0 && ktype[i] != 1) || !(C[i] > 0.0) ||
            !(knudsen[i] > 0.0))
            return FKS_ERR_INVALID_ARG;
    }
    fks_batch* b = new (std::nothrow) fks_batch();
    if (!b) return FKS_ERR_OOM;
    b->nprob = nprob;
    b->fp64 = precision == FKS_FP64;
    b->dirs = *dirs;
    b->M = dirs->A1 * dirs->A2;
    b->n.assign(n, n + nprob);
    b->L.assign(L, L + nprob);
    b->ktype.assign(ktype, ktype + nprob);
    b->Ck.assign(C, C + nprob);
    b->kn.assign(knudsen, knudsen + nprob);
    b->tset.resize(nprob);
    fks_status st = FKS_OK;
    // table sets: one per distinct (n, L, kernel, C)
    for (int i = 0; i < nprob; ++i) {
        int found = -1;
        for (size_t t = 0; t < b->tsets.size(); ++t) {
            const TableSet& ts = b->tsets[t];
            if (ts.n == n[i] && ts.L == L[i] && ts.ktype == ktype[i] && ts.Ck == C[i]) found = (int)t;
        }
        if (found < 0) {
            TableSet ts;
            ts.n = n[i];
            ts.L = L[i];
            ts.ktype = ktype[i];
            ts.Ck = C[i];
            double P[25];
            projection_matrix(n[i], L[i], P);
            if (cudaMalloc(&ts.P, sizeof(P)) != cudaSuccess || cudaMemcpy(ts.P, P, sizeof(P), cudaMemcpyHostToDevice))
                st = alloc_failure();
            b->tsets.push_back(ts);
            found = (int)b->tsets.size() - 1;
        }
        b->tset[i] = found;
    }
    // classes by n, in increasing n
    long first = 0;
    for (int nv : {8, 16, 24, 32}) {
        BatchClass cl;
        cl.n = nv;
        for (int i = 0; i < nprob; ++i)
            if (n[i] == nv) cl.probs.push_back(i);
        if (cl.probs.empty()) continue;
        cl.first = first;
        first += (long)cl.probs.size();
        b->classes.push_back(cl);
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) st = FKS_ERR_CUDA;
    if (cudaMalloc(&b->d_flags, sizeof(int)) != cudaSuccess || cudaMemset(b->d_flags, 0, sizeof(int)) != cudaSuccess)
        st = alloc_failure();
    for (BatchClass& cl : b->classes) {
        if (st != FKS_OK) break;
        if (cudaStreamCreateWithFlags(&cl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&cl.done, cudaEventDisableTiming) != cudaSuccess) {
            st = FKS_ERR_CUDA;
            break;
        }
        st = batch_configure_class(b, cl, default_cluster_size(b->fp64, cl.n));
        if (st == FKS_OK) st = batch_build_class_tables(b, cl);
        if (st == FKS_OK && !b->fp64) st = batch_setup_escalation(b, cl);
    }
    if (st == FKS_OK && !b->fp64) {
        if (cudaMalloc(&b->esc_lists, sizeof(int) * nprob) != cudaSuccess ||
            cudaMalloc(&b->esc_counts, sizeof(int) * b->classes.size()) != cudaSuccess)
            st = alloc_failure();
        else if (cudaMemset(b->esc_counts, 0, sizeof(int) * b->classes.size()) != cudaSuccess)
            st = FKS_ERR_CUDA;
        b->esc_tol = 1e-5;   // the stated FP32 bound (relative L2 of Q)
    }
    if (st != FKS_OK) {
        std::fprintf(stderr, "fks_batch_init: %s\n", b->err.c_str());
        fks_batch_destroy(b);
        return st;
    }
    *out = b;
    return FKS_OK;
}

void fks_batch_destroy(fks_batch* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    for (GraphEntry& g : b->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (ItemSet& s : b->items) {
        cudaFree(s.d);
        cudaFree(s.d64);
    }
    for (TableSet& t : b->tsets) {
        cudaFree(t.tables);
        cudaFree(t.tables64);
        cudaFree(t.P);
    }
    cudaFree(b->esc_lists);
    cudaFree(b->esc_counts);
    for (BatchClass& cl : b->classes) {
        if (cl.stream) cudaStreamDestroy(cl.stream);
        if (cl.done) cudaEventDestroy(cl.done);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    cudaFree(b->d_flags);
    delete b;
}

const char* fks_batch_last_error(const fks_batch* b) { return b ? b->err.c_str() : "null batch"; }
long fks_batch_launch_count(const fks_batch* b) { return b ? b->launches : -1; }

int fks_batch_cluster_size(const fks_batch* b, int n) {
    if (!b) return -1;
    for (const BatchClass& cl : b->classes)
        if (cl.n == n) return cl.C;
    return -1;
}

int fks_batch_radix(const fks_batch* b, int n) {
    if (!b) return -1;
    for (const BatchClass& cl : b->classes)
        if (cl.n == n) return cl.var.radix;
    return -1;
}

fks_status fks_batch_set_cluster_size(fks_batch* b, int n, int C) { return fks_batch_set_schedule(b, n, C, 0); }

fks_status fks_batch_set_schedule(fks_batch* b, int n, int C, int radix) {
    if (!b) return FKS_ERR_INVALID_ARG;
    for (BatchClass& cl : b->classes) {
        if (cl.n != n) continue;
        if (cl.C == C && cl.var.radix == radix) return FKS_OK;
        cudaDeviceSynchronize();
        const bool retable = cl.C != C;
        fks_status st = batch_configure_class(b, cl, C, radix);
        if (st != FKS_OK) return st;
        if (retable) st = batch_build_class_tables(b, cl);
        if (st != FKS_OK) return st;
        // descriptors and graphs hold table pointers: rebuild them on demand
        for (GraphEntry& g : b->graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        b->graphs.clear();
        for (ItemSet& s : b->items) {
            cudaFree(s.d);
            cudaFree(s.d64);
        }
        b->items.clear();
        return FKS_OK;
    }
    return bfail(b, FKS_ERR_INVALID_ARG, "no problem of this n in the batch");
}

static fks_status batch_check_ptrs(fks_batch* b, const void* const* f, void* const* o) {
    if (!f || !o) return bfail(b, FKS_ERR_INVALID_ARG, "null pointer array");
    for (int i = 0; i < b->nprob; ++i)
        if (!f[i] || !o[i] || f[i] == o[i] || !aligned16(f[i]) || !aligned16(o[i]))
            return bfail(b, FKS_ERR_INVALID_ARG, "problem arrays must be distinct 16-byte aligned device pointers");
    return FKS_OK;
}

fks_status fks_batch_collide(fks_batch* b, const void* const* f, void* const* Q, void* stream) {
    if (!b) return FKS_ERR_INVALID_ARG;
    fks_status st = batch_check_ptrs(b, f, Q);
    if (st != FKS_OK) return st;
    std::vector<double> zero(b->nprob, 0.0);
    BatchItem* d = nullptr;
    st = batch_items(b, f, Q, zero.data(), &d);
    if (st != FKS_OK) return st;
    return batch_launch(b, d, 0, (cudaStream_t)stream);
}

fks_status fks_batch_step(fks_batch* b, const void* const* f, void* const* f_out, const double* dt, void* stream) {
    if (!b || !dt) return FKS_ERR_INVALID_ARG;
    fks_status st = batch_check_ptrs(b, f, f_out);
    if (st != FKS_OK) return st;
    for (int i = 0; i < b->nprob; ++i)
        if (!std::isfinite(dt[i])) return bfail(b, FKS_ERR_INVALID_ARG, "dt must be finite");
    BatchItem* d = nullptr;
    st = batch_items(b, f, f_out, dt, &d);
    if (st != FKS_OK) return st;
    return batch_launch(b, d, 1, (cudaStream_t)stream);
}

fks_status fks_batch_run(fks_batch* b, void* const* fa, void* const* fb, const double* dt, int nsteps, void* stream) {
    if (!b || !dt || nsteps < 1) return FKS_ERR_INVALID_ARG;
    fks_status st = batch_check_ptrs(b, fa, fb);
    if (st != FKS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    GraphEntry* g = nullptr;
    for (GraphEntry& e : b->graphs) {
        bool same = e.nsteps == nsteps;
        for (int i = 0; i < b->nprob && same; ++i) same = e.a[i] == fa[i] && e.b[i] == fb[i] && e.dt[i] == dt[i];
        if (same) g = &e;
    }
    if (!g) {
        BatchItem *ab = nullptr, *ba = nullptr;
        st = batch_items(b, fa, fb, dt, &ab);
        if (st == FKS_OK) st = batch_items(b, fb, fa, dt, &ba);
        if (st != FKS_OK) return st;
        // capture on a private stream so that the caller's stream can be the legacy one
        cudaStream_t cap = nullptr;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return bfail(b, FKS_ERR_CUDA, "capture stream");
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        for (int k = 0; k < nsteps && e == cudaSuccess && st == FKS_OK; ++k) st = batch_launch(b, (k % 2) ? ba : ab, 1, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess || e2 != cudaSuccess || st != FKS_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st != FKS_OK ? st : bfail(b, FKS_ERR_CUDA, "graph capture");
        }
        GraphEntry ge;
        ge.a.assign(fa, fa + b->nprob);
        ge.b.assign(fb, fb + b->nprob);
        ge.dt.assign(dt, dt + b->nprob);
        ge.nsteps = nsteps;
        e = cudaGraphInstantiate(&ge.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bfail(b, FKS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        b->graphs.push_back(ge);
        g = &b->graphs.back();
    }
    cudaError_t e = cudaGraphLaunch(g->exec, s);
    if (e != cudaSuccess) return bfail(b, FKS_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    return FKS_OK;
}

fks_status fks_batch_set_escalation(fks_batch* b, double tol) {
    if (!b) return FKS_ERR_INVALID_ARG;
    if (!(tol >= 0.0) || !std::isfinite(tol)) return bfail(b, FKS_ERR_INVALID_ARG, "tol must be finite and >= 0");
    if (tol > 0.0 && b->fp64) return bfail(b, FKS_ERR_UNSUPPORTED, "FP64 batches have no escalation tier");
    cudaDeviceSynchronize();
    // captured graphs hold the launches of the old setting
    for (GraphEntry& g : b->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
    b->esc_tol = tol;
    return FKS_OK;
}

fks_status fks_batch_get_escalation(const fks_batch* b, double* tol, long* count) {
    if (!b) return FKS_ERR_INVALID_ARG;
    if (tol) *tol = b->esc_tol;
    if (count) {
        *count = 0;
        if (b->esc_counts) {
            std::vector<int> h(b->classes.size());
            if (cudaMemcpy(h.data(), b->esc_counts, sizeof(int) * h.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
                return FKS_ERR_CUDA;
            for (int v : h) *count += v;
        }
    }
    return FKS_OK;
}

fks_status fks_batch_check(fks_batch* b, void* stream, int* bits) {
    if (!b) return FKS_ERR_INVALID_ARG;
    int h = 0;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess ||
        cudaMemcpy(&h, b->d_flags, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(b->d_flags, 0, sizeof(int)) != cudaSuccess)
        return bfail(b, FKS_ERR_CUDA, "flag read");
    if (bits) *bits = h;
    if (h & 1) return bfail(b, FKS_ERR_NUMERIC, "non-finite value written");
    if (h & 8) return bfail(b, FKS_ERR_TIMEOUT, "a bulk copy did not complete in time");
    return FKS_OK;
}

}  // extern "C"
