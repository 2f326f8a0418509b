// api.cpp -- the C ABI of libqsim (declared in include/qsim.h).
//
// Host side only: argument validation, the lazy gate queue, planning and the
// dispatch of device work onto the handle's stream.  Every arithmetic step
// on amplitudes runs in the CUDA kernels (gate_kernels.cu,
// tmem_block_kernel.cu, diag_kernels.cu, perm_kernels.cu,
// reduce_kernels.cu).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

int set_err(qsim *s, int code, const std::string &msg) {
    if (s) s->err = msg;
    return code;
}

int cuda_err(qsim *s, cudaError_t e, const char *where) {
    if (e == cudaSuccess) return QSIM_OK;
    if (s) s->err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? QSIM_ENOMEM : QSIM_ECUDA;
}

namespace {

constexpr size_t kPinnedBytes = 64u << 10;

int validate_qubits(qsim *s, const int *a, int na, const int *b, int nb, uint64_t *ma, uint64_t *mb) {
    uint64_t seen = 0;
    *ma = *mb = 0;
    for (int j = 0; j < na; ++j) {
        if (a[j] < 0 || a[j] >= s->n) return set_err(s, QSIM_ERANGE, "qubit index out of range");
        if ((seen >> a[j]) & 1ull) return set_err(s, QSIM_EDUP, "qubit named twice");
        seen |= 1ull << a[j];
        *ma |= 1ull << a[j];
    }
    for (int j = 0; j < nb; ++j) {
        if (b[j] < 0 || b[j] >= s->n) return set_err(s, QSIM_ERANGE, "qubit index out of range");
        if ((seen >> b[j]) & 1ull) return set_err(s, QSIM_EDUP, "qubit named twice");
        seen |= 1ull << b[j];
        *mb |= 1ull << b[j];
    }
    return QSIM_OK;
}

// Start a new norm-control chain of the tensor-core block passes (see
// tmem_block_kernel.cu): the next block pass applies no correction and the
// chain steers to `target` (<= 0: that pass's input norm).  Called wherever
// the norm legitimately changes or becomes unknown to the device records.
void norm_anchor(qsim *s, double target) {
    s->norm_chain = false;
    s->norm_target = target;
}

// max |U U^dag - I| <= 1e-9: the gate keeps the norm
bool is_unitary(const GateRec &g) {
    const int D = 1 << g.t;
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c) {
            cd acc(0.0, 0.0);
            for (int k = 0; k < D; ++k) acc += g.m[(size_t)r * D + k] * std::conj(g.m[(size_t)c * D + k]);
            if (std::abs(acc - cd(r == c ? 1.0 : 0.0, 0.0)) > 1e-9) return false;
        }
    return true;
}

int classify(const GateRec &g) {
    if (g.t != 1) return GK_DENSE;
    const cd *m = g.m.data();
    if (m[1] == 0.0 && m[2] == 0.0) return m[0] == 1.0 ? GK_PHASE : GK_DIAG1;
    if (m[0] == 0.0 && m[3] == 0.0 && m[1] == 1.0 && m[2] == 1.0) return GK_X;
    return GK_DENSE;
}

double gate_bytes(const qsim *s, const GateRec &g) {
    const double b = (double)amp_bytes(s);
    int fixed = (int)g.controls.size();
    if (g.kind == GK_PHASE) fixed += 1;
    return 2.0 * b * std::ldexp(1.0, s->n - fixed);
}

const char *kClassName[KC_COUNT] = {"gate_dense", "gate_phase", "gate_diag",  "gate_x",  "block_tc",
                                    "block_dense", "block_diag", "block_tc6", "permute", "permute_cycles",
                                    "permute_cycles_bulk", "product"};

int harvest(qsim *s) {
    if (s->pending.empty()) return QSIM_OK;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_err(s, e, "stream synchronize");
    for (const auto &p : s->pending) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, s->ev_pool[p.ev], s->ev_pool[p.ev + 1]);
        if (e != cudaSuccess) return cuda_err(s, e, "event elapsed");
        auto &c = s->class_time[p.cls];
        c.launches++;
        c.ms += ms;
        c.bytes += p.bytes;
        if (p.feat >= 0) {
            s->item_feats.insert(s->item_feats.end(), s->pending_feats.begin() + p.feat,
                                 s->pending_feats.begin() + p.feat + kFeatures);
            // the item's cost: device time, or host time where the host is slower
            s->item_ms.push_back(ms > p.host_ms ? ms : p.host_ms);
        }
    }
    s->pending.clear();
    s->pending_feats.clear();
    s->ev_used = 0;
    return QSIM_OK;
}

// Record an event on the stream; returns its pool index.
int record_event(qsim *s, size_t *idx) {
    if (s->ev_used == s->ev_pool.size()) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return cuda_err(s, e, "event create");
        s->ev_pool.push_back(ev);
    }
    *idx = s->ev_used++;
    return cuda_err(s, cudaEventRecord(s->ev_pool[*idx], s->stream), "event record");
}

int gate_class(const GateRec &g) {
    switch (g.kind) {
    case GK_PHASE: return KC_PHASE;
    case GK_DIAG1: return KC_DIAG;
    case GK_X: return KC_X;
    default: return KC_DENSE;
    }
}

// Widest block the executors take: 6-qubit blocks exist only as the
// complex64 tensor-core kernel (tiles of 2^13 amplitudes); elsewhere kmax 6
// plans 5-qubit blocks.
int block_kmax(const qsim *s) {
    if (s->kmax == 6 && (s->prec != QSIM_C64 || !s->tc_enabled || s->n < 13)) return 5;
    return s->kmax;
}

// Launch one planned item.  With profiling: events around it; in mode 2
// also its features and its host time (building the block matrix, the
// operand record, staging and launching), for the cost model.
int execute_item(qsim *s, const PlanItem &it) {
    const auto h0 = std::chrono::steady_clock::now();
    int rc;
    size_t ev0 = 0, ev1 = 0;
    // with profiling on, an NVTX range per planned item (visible in a
    // timeline profiler next to its kernel)
    struct Range {
        bool on;
        Range(bool o, const PlanItem &it) : on(o) {
            if (on)
                nvtxRangePushA(!it.fused        ? "gate"
                               : it.diag_block  ? "diag block"
                               : it.perm_block  ? "perm block"
                               : it.prod_block  ? "product"
                                                : "dense block");
        }
        ~Range() {
            if (on) nvtxRangePop();
        }
    } range(s->profiling, it);
    // a non-unitary gate changes the norm: no correction across it
    bool unitary = true;
    for (int gi : it.members) unitary = unitary && s->queue[gi].unitary;
    if (!unitary) norm_anchor(s, -1.0);
    if (s->profiling) {
        if (s->pending.size() >= 4096 && (rc = harvest(s))) return rc;
        if ((rc = record_event(s, &ev0))) return rc;
    }
    int cls;
    double bytes;
    if (!it.fused) {
        const GateRec &g = s->queue[it.gate];
        rc = launch_gate_plain(s, g);
        bytes = gate_bytes(s, g);
        cls = gate_class(g);
    } else if (it.diag_block) {
        cls = KC_BLOCK_DIAG;
        rc = launch_block_diag(s, it.dmask, it.dtab.data());
        bytes = 2.0 * (double)amp_bytes(s) * std::ldexp(1.0, s->n);
    } else if (it.prod_block) {
        int npasses = 0;
        cls = KC_PRODUCT;
        rc = launch_product(s, it.qmask_prod, it.pm.data(), &npasses);
        bytes = 2.0 * (double)amp_bytes(s) * std::ldexp(1.0, s->n) * npasses;
        s->stats.passes += npasses > 0 ? npasses - 1 : 0;  // one is counted below
    } else if (it.perm_block) {
        int qubits[64], m = 0, kind = 0;
        for (int b = 0; b < s->n; ++b)
            if ((it.pmask >> b) & 1ull) qubits[m++] = b;
        rc = launch_permutation(s, it.ptab.data(), qubits, m, it.pmask, 0, &kind);
        cls = kind == 2 ? KC_PERMUTE_BULK : kind == 1 ? KC_PERMUTE_CYCLES : KC_PERMUTE;
        bytes = 2.0 * (double)amp_bytes(s) * std::ldexp(1.0, s->n);
    } else {
        rc = QSIM_ENOTSUP;
        cls = KC_BLOCK_TC;
        if (it.k == 6) {
            cls = KC_BLOCK_TC6;
            rc = launch_block_tmem(s, it.qubits, 6, it.m.data());
        } else if (s->prec == QSIM_C64 && it.k >= 4)
            rc = launch_block_tc(s, it.qubits, it.k, it.m.data());
        if (rc == QSIM_ENOTSUP) {
            cls = KC_BLOCK_DENSE;
            rc = launch_block_dense(s, it.qubits, it.k, it.m.data());
        }
        bytes = 2.0 * (double)amp_bytes(s) * std::ldexp(1.0, s->n);
    }
    if (rc) return rc;
    if (!unitary) norm_anchor(s, -1.0);
    const auto h1 = std::chrono::steady_clock::now();
    s->stats.alg_bytes += bytes;
    if (s->profiling) {
        if ((rc = record_event(s, &ev1))) return rc;
        (void)ev1;
        long feat = -1;
        if (s->record_items) {
            feat = (long)s->pending_feats.size();
            s->pending_feats.resize(s->pending_feats.size() + kFeatures);
            item_features(it, s->queue, s->n, s->prec, s->tc_enabled, s->c128_df, &s->pending_feats[feat]);
        }
        const double host_ms = it.host_ms + std::chrono::duration<double, std::milli>(h1 - h0).count();
        s->pending.push_back({cls, ev0, bytes, feat, (float)host_ms});
    }
    s->stats.passes++;
    s->stats.amp_updates += it.amp_updates;
    return QSIM_OK;
}

int execute_plan(qsim *s, const std::vector<PlanItem> &plan) {
    for (const PlanItem &it : plan)
        if (const int rc = execute_item(s, it)) return rc;
    return QSIM_OK;
}

int flush(qsim *s) {
    if (s->queue.empty()) return QSIM_OK;
    int rc;
    const std::vector<GateRec> &q = s->queue;
    MlpChoice ch;
    if (s->fusion == QSIM_FUSE_MLP && s->cost.loaded()) {
        plan_mlp(q, s->n, s->prec, s->tc_enabled, s->c128_df, s->perm_blocks, block_kmax(s), s->cost, ch);
        s->last_plan_predicted_ms = ch.predicted_ms;
    }
    if (s->fusion == QSIM_FUSE_NONE || (s->fusion == QSIM_FUSE_MLP && s->cost.loaded() && ch.kmax == 1)) {
        std::vector<PlanItem> plan;
        plan_none(q, s->n, plan);
        rc = execute_plan(s, plan);
    } else if (s->fusion == QSIM_FUSE_MLP && s->cost.loaded()) {
        // the chosen plan, regenerated item by item and launched as it forms
        size_t idx = 0;
        rc = plan_greedy_each(
            q, s->n, ch.kmax,
            [&](PlanItem &it) {
                const bool fuse = idx < ch.fuse.size() && ch.fuse[idx];
                ++idx;
                if (!it.fused) return execute_item(s, it);
                if (fuse) {
                    block_matrix(q, it);
                    return execute_item(s, it);
                }
                for (int gi : it.members)
                    if (const int r = execute_item(s, single_item(q, s->n, gi))) return r;
                return 0;
            },
            kMaxDiagQubits, false, s->perm_blocks ? perm_min_width(s->prec, ch.kmax) : 0);
    } else {
        // greedy: each block is launched as soon as it is formed, so the
        // host's planning of the next blocks overlaps the device's work.
        // Where planning the queue twice costs less than a tenth of one pass
        // over the state (about 1 us per gate against 2^n amplitudes read
        // and written at some 6.5 TB/s), both dense tie rules are planned
        // first and the one with fewer passes is launched
        const bool prod = s->prod_passes && s->prec == QSIM_C64 && s->n >= 12;
        const int perm_min = s->perm_blocks ? perm_min_width(s->prec, block_kmax(s)) : 0;
        const int prod_min = prod ? block_kmax(s) + 1 : 0;
        const double pass_us = 2.0 * (double)amp_bytes(s) * std::ldexp(1.0, s->n) / 6.5e6;
        int tie = 0;
        if (2.0 * (double)q.size() < 0.1 * pass_us) {
            std::vector<PlanItem> p0, p1;
            plan_greedy(q, s->n, block_kmax(s), p0, kMaxDiagQubits, false, perm_min, prod_min, 0);
            plan_greedy(q, s->n, block_kmax(s), p1, kMaxDiagQubits, false, perm_min, prod_min, 1);
            auto passes = [](const std::vector<PlanItem> &p) {
                size_t c = 0;
                for (const PlanItem &it : p) c += it.prod_block ? (size_t)product_pass_count(it.qmask_prod) : 1;
                return c;
            };
            if (passes(p1) < passes(p0)) tie = 1;
        }
        rc = plan_greedy_each(
            s->queue, s->n, block_kmax(s), [s](PlanItem &it) { return execute_item(s, it); }, kMaxDiagQubits, true,
            perm_min, prod_min, tie);
    }
    s->queue.clear();
    return rc;
}

bool is_finite(double x) { return std::isfinite(x); }

}  // namespace

int stage_operand(qsim *s, const void *data, size_t bytes, unsigned char **dev) {
    const size_t need = (bytes + 255) & ~(size_t)255;
    if (need > kWsRingBytes) return set_err(s, QSIM_EINVAL, "block operand too large");
    if (!s->stage_host) {
        if (cudaMallocHost((void **)&s->stage_host, kWsRingBytes) != cudaSuccess) {
            cudaGetLastError();
            s->stage_host = nullptr;
            return set_err(s, QSIM_ENOMEM, "pinned staging buffer");
        }
        s->stage_cursor = 0;
    }
    if (s->stage_cursor + need > kWsRingBytes) {
        // every earlier copy out of the staging buffer must have run
        cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_err(s, e, "stream synchronize");
        s->stage_cursor = 0;
    }
    std::memcpy(s->stage_host + s->stage_cursor, data, bytes);
    unsigned char *d = (unsigned char *)s->ws + kWsRing + s->stage_cursor;
    cudaError_t e = cudaMemcpyAsync(d, s->stage_host + s->stage_cursor, bytes, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_err(s, e, "operand copy");
    s->stage_cursor += need;
    *dev = d;
    return QSIM_OK;
}

int check_device_errors(qsim *s) {
    unsigned int *flag = (unsigned int *)((char *)s->ws + kWsErr);
    cudaError_t e = cudaMemcpyAsync(s->pinned, flag, sizeof(unsigned int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_err(s, e, "error flag read");
    unsigned int v;
    std::memcpy(&v, s->pinned, sizeof(v));
    if (v) {
        cudaMemsetAsync(flag, 0, sizeof(unsigned int), s->stream);
        return set_err(s, QSIM_ETIMEOUT, "a bounded device wait gave up (flag " + std::to_string(v) + ")");
    }
    return QSIM_OK;
}

extern "C" {

int sim_workspace_bytes(int n, int precision, size_t *bytes) {
    if (!bytes || n < 1 || n > 36 || (precision != QSIM_C128 && precision != QSIM_C64)) return QSIM_EINVAL;
    *bytes = kWsTotal;
    return QSIM_OK;
}

int sim_create(int n, int precision, const qsim_opts *opts, qsim **out) {
    if (!out) return QSIM_EINVAL;
    *out = nullptr;
    if (n < 1 || n > 36) return QSIM_EINVAL;
    if (precision != QSIM_C128 && precision != QSIM_C64) return QSIM_EINVAL;
    qsim_opts o{};
    if (opts) o = *opts;
    if (o.fusion < QSIM_FUSE_NONE || o.fusion > QSIM_FUSE_MLP) return QSIM_EINVAL;
    if (o.kmax == 0) o.kmax = 6;
    if (o.kmax < 1 || o.kmax > 6) return QSIM_EINVAL;
    qsim *s = new (std::nothrow) qsim();
    if (!s) return QSIM_ENOMEM;
    s->n = n;
    s->prec = precision;
    s->fusion = o.fusion;
    s->kmax = o.kmax;
    if (o.tc_terms != 0 && o.tc_terms != 3 && o.tc_terms != 5) {
        delete s;
        return QSIM_EINVAL;
    }
    s->tc_terms = o.tc_terms == 5 ? 5 : 3;
    s->tc_enabled = o.no_tensor_cores == 0;
    s->norm_tracking = o.no_norm_tracking == 0;
    s->c128_df = o.c128_double_float != 0;
    s->perm_blocks = o.no_permutation_blocks == 0;
    s->prod_passes = o.no_product_passes == 0;
    s->stream = (cudaStream_t)o.stream;
    if (o.device >= 0) {
        if (cudaSetDevice(o.device) != cudaSuccess) {
            delete s;
            return QSIM_ECUDA;
        }
    }
    cudaGetDevice(&s->device);
    if (cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess || s->sms < 1) {
        cudaGetLastError();
        delete s;
        return QSIM_ECUDA;
    }
    const size_t need = amp_bytes(s) << n;
    int rc = QSIM_OK;
    if (o.state) {
        if (o.state_bytes < need || ((uintptr_t)o.state & 255u)) rc = QSIM_EINVAL;
        s->state = o.state;
    } else {
        cudaError_t e = cudaMalloc(&s->state, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s->state = nullptr;
            rc = QSIM_ENOMEM;
        } else {
            s->own_state = true;
        }
    }
    if (!rc) {
        if (o.workspace) {
            if (o.workspace_bytes < kWsTotal || ((uintptr_t)o.workspace & 255u)) rc = QSIM_EINVAL;
            s->ws = o.workspace;
            s->ws_bytes = o.workspace_bytes;
        } else {
            cudaError_t e = cudaMalloc(&s->ws, kWsTotal);
            if (e != cudaSuccess) {
                cudaGetLastError();
                s->ws = nullptr;
                rc = QSIM_ENOMEM;
            } else {
                s->own_ws = true;
                s->ws_bytes = kWsTotal;
            }
        }
    }
    if (!rc && cudaMallocHost((void **)&s->pinned, kPinnedBytes) != cudaSuccess) {
        cudaGetLastError();
        s->pinned = nullptr;
        rc = QSIM_ENOMEM;
    }
    if (!rc) rc = cuda_err(s, cudaMemsetAsync((char *)s->ws + kWsErr, 0, kWsErrBytes, s->stream), "clear flags");
    if (!rc) rc = launch_set_basis(s, 0);
    if (rc) {
        sim_destroy(s);
        return rc;
    }
    *out = s;
    return QSIM_OK;
}

int sim_destroy(qsim *s) {
    if (!s) return QSIM_OK;
    if (s->stream || s->state) cudaStreamSynchronize(s->stream);
    if (s->own_state && s->state) cudaFree(s->state);
    if (s->own_ws && s->ws) cudaFree(s->ws);
    if (s->pinned) cudaFreeHost(s->pinned);
    if (s->stage_host) cudaFreeHost(s->stage_host);
    for (cudaEvent_t ev : s->ev_pool) cudaEventDestroy(ev);
    delete s;
    return QSIM_OK;
}

int sim_reset(qsim *s, uint64_t basis) {
    if (!s) return QSIM_EINVAL;
    if (basis >> s->n) return set_err(s, QSIM_ERANGE, "basis state out of range");
    s->queue.clear();
    norm_anchor(s, 1.0);
    return launch_set_basis(s, basis);
}

int sim_apply(qsim *s, const double *matrix, const int *targets, int t, const int *controls, int c) {
    if (!s) return QSIM_EINVAL;
    if (!matrix || !targets || t < 1 || t > 5 || c < 0 || (c > 0 && !controls))
        return set_err(s, QSIM_EINVAL, "bad gate arguments");
    if (t + c > s->n) return set_err(s, QSIM_ERANGE, "more qubits than the register has");
    GateRec g;
    int rc = validate_qubits(s, targets, t, controls, c, &g.tmask, &g.cmask);
    if (rc) return rc;
    const int D = 1 << t;
    for (int i = 0; i < 2 * D * D; ++i)
        if (!is_finite(matrix[i])) return set_err(s, QSIM_ENONFINITE, "non-finite matrix entry");
    g.t = t;
    for (int j = 0; j < t; ++j) g.targets[j] = targets[j];
    g.controls.assign(controls, controls + c);
    g.m.resize((size_t)D * D);
    for (int i = 0; i < D * D; ++i) g.m[i] = cd(matrix[2 * i], matrix[2 * i + 1]);
    g.kind = classify(g);
    g.unitary = is_unitary(g);
    g.perm = perm_map(g, g.pmap);
    g.diag = true;
    for (int r = 0; r < D && g.diag; ++r)
        for (int c = 0; c < D; ++c)
            if (r != c && g.m[(size_t)r * D + c] != 0.0) {
                g.diag = false;
                break;
            }
    s->queue.push_back(std::move(g));
    s->stats.gates++;
    return QSIM_OK;
}

int sim_flush(qsim *s) {
    if (!s) return QSIM_EINVAL;
    return flush(s);
}

int sim_apply_permutation(qsim *s, const uint64_t *perm, const int *qubits, int m, const int *controls, int c) {
    if (!s) return QSIM_EINVAL;
    if (!perm || !qubits || m < 1 || m > 12 || c < 0 || (c > 0 && !controls))
        return set_err(s, QSIM_EINVAL, "bad permutation arguments");
    if (m + c > s->n) return set_err(s, QSIM_ERANGE, "more qubits than the register has");
    uint64_t qmask, cmask;
    int rc = validate_qubits(s, qubits, m, controls, c, &qmask, &cmask);
    if (rc) return rc;
    const uint64_t D = 1ull << m;
    std::vector<char> seen(D, 0);
    for (uint64_t v = 0; v < D; ++v) {
        if (perm[v] >= D || seen[perm[v]]) return set_err(s, QSIM_EINVAL, "permutation is not a bijection");
        seen[perm[v]] = 1;
    }
    if ((rc = flush(s))) return rc;
    size_t ev0 = 0, ev1 = 0;
    if (s->profiling && (rc = record_event(s, &ev0))) return rc;
    int kind = 0;
    rc = launch_permutation(s, perm, qubits, m, qmask, cmask, &kind);
    if (rc) return rc;
    const double bytes = 2.0 * (double)amp_bytes(s) * std::ldexp(1.0, s->n - c);
    if (s->profiling) {
        if ((rc = record_event(s, &ev1))) return rc;
        s->pending.push_back({kind == 2 ? KC_PERMUTE_BULK : kind == 1 ? KC_PERMUTE_CYCLES : KC_PERMUTE, ev0, bytes,
                              -1, 0.f});
    }
    s->stats.passes++;
    s->stats.amp_updates += std::ldexp(1.0, s->n - c);
    s->stats.alg_bytes += bytes;
    return QSIM_OK;
}

int sim_prob(qsim *s, int qubit, double *p1) {
    if (!s || !p1) return QSIM_EINVAL;
    if (qubit < 0 || qubit >= s->n) return set_err(s, QSIM_ERANGE, "qubit index out of range");
    int rc = flush(s);
    if (rc) return rc;
    return run_masked_sum(s, 1ull << qubit, 1ull << qubit, p1);
}

int sim_probs_all(qsim *s, double *p1, double *norm2) {
    if (!s || !p1) return QSIM_EINVAL;
    int rc = flush(s);
    if (rc) return rc;
    return run_probs_all(s, p1, norm2);
}

int sim_measure(qsim *s, int qubit, double u, int *outcome, double *p_outcome) {
    if (!s || !outcome) return QSIM_EINVAL;
    if (qubit < 0 || qubit >= s->n) return set_err(s, QSIM_ERANGE, "qubit index out of range");
    if (!(u >= 0.0 && u < 1.0)) return set_err(s, QSIM_EINVAL, "draw outside [0,1)");
    int rc = flush(s);
    if (rc) return rc;
    double s0, s1;
    rc = run_split_sum(s, qubit, &s0, &s1);
    if (rc) return rc;
    const int b = (u * (s0 + s1) < s0) ? 0 : 1;
    const double p = b ? s1 : s0;
    if (!(p > 0.0)) return set_err(s, QSIM_EZEROPROB, "measured outcome has probability 0");
    rc = run_collapse_mask(s, 1ull << qubit, (uint64_t)b << qubit, 1.0 / std::sqrt(p));
    if (rc) return rc;
    norm_anchor(s, 1.0);
    *outcome = b;
    // the probability that decided the outcome (relative to the norm)
    if (p_outcome) *p_outcome = p / (s0 + s1);
    return QSIM_OK;
}

int sim_collapse(qsim *s, const int *qubits, int m, const int *bits, double *p) {
    if (!s || m < 1 || !qubits || !bits) return QSIM_EINVAL;
    uint64_t mask, dummy;
    int rc = validate_qubits(s, qubits, m, nullptr, 0, &mask, &dummy);
    if (rc) return rc;
    uint64_t value = 0;
    for (int j = 0; j < m; ++j) {
        if (bits[j] != 0 && bits[j] != 1) return set_err(s, QSIM_EINVAL, "bit values must be 0 or 1");
        if (bits[j]) value |= 1ull << qubits[j];
    }
    rc = flush(s);
    if (rc) return rc;
    double pv;
    rc = run_masked_sum(s, mask, value, &pv);
    if (rc) return rc;
    if (p) *p = pv;
    if (!(pv > 0.0)) return set_err(s, QSIM_EZEROPROB, "projection has probability 0");
    rc = run_collapse_mask(s, mask, value, 1.0 / std::sqrt(pv));
    if (!rc) norm_anchor(s, 1.0);
    return rc;
}

int sim_measure_all(qsim *s, double u, uint64_t *outcome) {
    if (!s || !outcome) return QSIM_EINVAL;
    if (!(u >= 0.0 && u < 1.0)) return set_err(s, QSIM_EINVAL, "draw outside [0,1)");
    int rc = flush(s);
    if (rc) return rc;
    rc = run_measure_all(s, u, outcome);
    if (!rc) norm_anchor(s, 1.0);
    return rc;
}

int sim_expect(qsim *s, const qsim_pauli *terms, int nterms, double *out) {
    if (!s || !out || nterms < 0 || (nterms > 0 && !terms)) return QSIM_EINVAL;
    const uint64_t lim = s->n >= 64 ? ~0ull : ((1ull << s->n) - 1);
    for (int k = 0; k < nterms; ++k) {
        if ((terms[k].xmask & ~lim) || (terms[k].zmask & ~lim))
            return set_err(s, QSIM_ERANGE, "Pauli mask names a qubit out of range");
        if (!is_finite(terms[k].coeff)) return set_err(s, QSIM_ENONFINITE, "non-finite coefficient");
    }
    int rc = flush(s);
    if (rc) return rc;
    if (nterms == 0) {
        *out = 0.0;
        return QSIM_OK;
    }
    return run_expect(s, terms, nterms, out);
}

int sim_get_amplitudes(qsim *s, uint64_t offset, uint64_t count, double *out) {
    if (!s || (!out && count)) return QSIM_EINVAL;
    const uint64_t N = 1ull << s->n;
    if (offset > N || count > N - offset) return set_err(s, QSIM_ERANGE, "amplitude range out of bounds");
    int rc = flush(s);
    if (rc) return rc;
    if (!count) return QSIM_OK;
    cudaError_t e;
    if ((rc = check_device_errors(s))) return rc;
    if (s->prec == QSIM_C128) {
        e = cudaMemcpyAsync(out, (const char *)s->state + offset * 16, count * 16, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        return cuda_err(s, e, "amplitude copy");
    }
    std::vector<float> tmp;
    try {
        tmp.resize(2 * count);
    } catch (...) {
        return set_err(s, QSIM_ENOMEM, "host buffer");
    }
    e = cudaMemcpyAsync(tmp.data(), (const char *)s->state + offset * 8, count * 8, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_err(s, e, "amplitude copy");
    for (uint64_t i = 0; i < 2 * count; ++i) out[i] = (double)tmp[i];
    return QSIM_OK;
}

int sim_set_amplitudes(qsim *s, uint64_t offset, uint64_t count, const double *in) {
    if (!s || (!in && count)) return QSIM_EINVAL;
    const uint64_t N = 1ull << s->n;
    if (offset > N || count > N - offset) return set_err(s, QSIM_ERANGE, "amplitude range out of bounds");
    for (uint64_t i = 0; i < 2 * count; ++i)
        if (!is_finite(in[i])) return set_err(s, QSIM_ENONFINITE, "non-finite amplitude");
    int rc = flush(s);
    if (rc) return rc;
    if (!count) return QSIM_OK;
    norm_anchor(s, -1.0);
    cudaError_t e;
    if (s->prec == QSIM_C128) {
        e = cudaMemcpyAsync((char *)s->state + offset * 16, in, count * 16, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        return cuda_err(s, e, "amplitude copy");
    }
    std::vector<float> tmp;
    try {
        tmp.resize(2 * count);
    } catch (...) {
        return set_err(s, QSIM_ENOMEM, "host buffer");
    }
    for (uint64_t i = 0; i < 2 * count; ++i) tmp[i] = (float)in[i];
    e = cudaMemcpyAsync((char *)s->state + offset * 8, tmp.data(), count * 8, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return cuda_err(s, e, "amplitude copy");
}

int sim_state_ptr(qsim *s, void **dev_ptr) {
    if (!s || !dev_ptr) return QSIM_EINVAL;
    int rc = flush(s);
    if (rc) return rc;
    // the caller may write through the pointer
    norm_anchor(s, -1.0);
    *dev_ptr = s->state;
    return QSIM_OK;
}

int sim_set_stream(qsim *s, void *stream) {
    if (!s) return QSIM_EINVAL;
    int rc = flush(s);
    if (rc) return rc;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_err(s, e, "stream synchronize");
    s->stream = (cudaStream_t)stream;
    return QSIM_OK;
}

int sim_set_fusion(qsim *s, int mode, int kmax) {
    if (!s) return QSIM_EINVAL;
    if (mode < QSIM_FUSE_NONE || mode > QSIM_FUSE_MLP) return set_err(s, QSIM_EINVAL, "unknown fusion mode");
    if (kmax < 1 || kmax > 6) return set_err(s, QSIM_EINVAL, "kmax outside 1..6");
    int rc = flush(s);
    if (rc) return rc;
    s->fusion = mode;
    s->kmax = kmax;
    return QSIM_OK;
}

int sim_get_stats(const qsim *s, qsim_stats *out) {
    if (!s || !out) return QSIM_EINVAL;
    *out = s->stats;
    return QSIM_OK;
}

int sim_reset_stats(qsim *s) {
    if (!s) return QSIM_EINVAL;
    s->stats = qsim_stats{};
    return QSIM_OK;
}

int sim_set_profiling(qsim *s, int on) {
    if (!s) return QSIM_EINVAL;
    int rc = flush(s);
    if (rc) return rc;
    if ((rc = harvest(s))) return rc;
    s->profiling = on != 0;
    s->record_items = on == 2;
    s->item_feats.clear();
    s->item_ms.clear();
    for (auto &c : s->class_time) c = qsim::ClassTime{};
    return QSIM_OK;
}

int sim_get_kernel_times(qsim *s, qsim_kernel_time *rows, int max_rows, int *nrows) {
    if (!s || !nrows || (max_rows > 0 && !rows)) return QSIM_EINVAL;
    int rc = flush(s);
    if (rc) return rc;
    if ((rc = harvest(s))) return rc;
    int k = 0;
    for (int c = 0; c < KC_COUNT; ++c) {
        if (!s->class_time[c].launches) continue;
        if (k < max_rows) {
            std::memset(&rows[k], 0, sizeof(rows[k]));
            std::strncpy(rows[k].name, kClassName[c], sizeof(rows[k].name) - 1);
            rows[k].launches = s->class_time[c].launches;
            rows[k].total_ms = s->class_time[c].ms;
            rows[k].alg_bytes = s->class_time[c].bytes;
        }
        ++k;
    }
    *nrows = k;
    return QSIM_OK;
}

int sim_get_item_times(qsim *s, float *feats, float *ms, int max_items, int *nitems) {
    if (!s || !nitems || (max_items > 0 && (!feats || !ms))) return QSIM_EINVAL;
    int rc = flush(s);
    if (rc) return rc;
    if ((rc = harvest(s))) return rc;
    const int n = (int)s->item_ms.size();
    const int k = n < max_items ? n : max_items;
    if (k > 0) {
        std::memcpy(feats, s->item_feats.data(), sizeof(float) * kFeatures * k);
        std::memcpy(ms, s->item_ms.data(), sizeof(float) * k);
    }
    *nitems = n;
    if (k == n) {
        s->item_feats.clear();
        s->item_ms.clear();
    }
    return QSIM_OK;
}

int sim_set_cost_model(qsim *s, const float *params, int count, int hidden) {
    if (!s) return QSIM_EINVAL;
    if (count == 0) {
        s->cost = CostModel{};
        return QSIM_OK;
    }
    if (!params || hidden < 1 || hidden > kMaxHidden) return set_err(s, QSIM_EINVAL, "bad cost model");
    const long need = (long)hidden * kFeatures + hidden + (long)hidden * hidden + hidden + hidden + 1;
    if (count != need) return set_err(s, QSIM_EINVAL, "cost model size does not match hidden width");
    for (int i = 0; i < count; ++i)
        if (!std::isfinite(params[i])) return set_err(s, QSIM_ENONFINITE, "non-finite cost model parameter");
    s->cost.hidden = hidden;
    s->cost.p.assign(params, params + count);
    return QSIM_OK;
}

int sim_plan_stats(qsim *s, double *predicted_ms) {
    if (!s || !predicted_ms) return QSIM_EINVAL;
    *predicted_ms = s->last_plan_predicted_ms;
    return QSIM_OK;
}

const char *sim_last_error(const qsim *s) { return s ? s->err.c_str() : "null handle"; }

const char *qsim_build_info(void) { return "libqsim 0.1 sm_103a"; }

}  // extern "C"
