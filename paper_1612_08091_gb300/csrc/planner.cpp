// planner.cpp -- the lazy gate queue turned into device work.
//
// The paper's simulator buffers gates and executes them later ("lazy
// evaluation of gates", ProjectQ paper Sec. 4.3.2, Fig. 7 caption).  Here the
// buffered queue is either executed gate by gate (plan_none) or grouped into
// dense blocks of at most kmax qubits (plan_greedy), each executed as one
// pass over the state vector.
//
// plan_greedy works on the circuit's dependency structure, not on the raw
// gate order: gates on disjoint qubits commute, so a block may take any gate
// that is "ready" (every earlier gate on each of its qubits is already
// executed or inside the block).  Starting from the earliest ready gate, a
// block first absorbs every ready gate whose qubits it already covers, then
// grows by the ready gate that adds the fewest new qubits while it still
// fits in kmax, and repeats until nothing more fits.  The block's matrix is
// the ordered product of its gates, each embedded in the block's qubits, in
// FP64.  Runs of diagonal gates become diagonal blocks of up to 12 qubits
// (grown with a look-ahead: see the diagonal branch) and runs of
// permutation gates permutation blocks.  Gates on more than kmax qubits
// (e.g. a many-controlled Z) run alone with their specialised plain
// kernel.  Between such gates, a layer of
// one-qubit gates on more than kmax qubits (Grover's H and X layers, paper
// Appendix A) has nothing to fuse with: it becomes a product item, the 2x2
// product of each wire's gates, executed 12 qubits per pass.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <functional>

#include <cmath>

#include "internal.h"

void plan_none(const std::vector<GateRec> &q, int n, std::vector<PlanItem> &out) {
    out.clear();
    out.reserve(q.size());
    for (size_t i = 0; i < q.size(); ++i) {
        PlanItem it;
        it.fused = false;
        it.gate = (int)i;
        it.amp_updates = (double)(1ull << (n - (int)q[i].controls.size()));
        it.ngates = 1;
        it.members.push_back((int)i);
        out.push_back(std::move(it));
    }
}

namespace {

// Apply gate g to the 2^k x 2^k block matrix M (row-major, row/column bit j
// = qubit S[j]) from the left: M <- G M.  Row-oriented, so the inner loops
// run along contiguous rows: an X (with controls) swaps pairs of rows, a
// diagonal gate scales rows, a dense gate mixes each group of 2^t rows.
void apply_to_block(std::vector<cd> &M, int k, const int *S, const GateRec &g) {
    const int D = 1 << k;
    auto pos = [&](int qubit) {
        for (int j = 0; j < k; ++j)
            if (S[j] == qubit) return j;
        return -1;
    };
    int tm = 0, cm = 0;
    int spread[32];  // row offset of target pattern r (bit j of r -> bit pos(targets[j]))
    const int T = 1 << g.t;
    int tbits[5];
    for (int j = 0; j < g.t; ++j) {
        tbits[j] = 1 << pos(g.targets[j]);
        tm |= tbits[j];
    }
    for (int r = 0; r < T; ++r) {
        spread[r] = 0;
        for (int j = 0; j < g.t; ++j)
            if ((r >> j) & 1) spread[r] |= tbits[j];
    }
    for (int c : g.controls) cm |= 1 << pos(c);
    double *m = reinterpret_cast<double *>(M.data());  // interleaved (re, im)
    const size_t row = 2 * (size_t)D;                  // doubles per row
    if (g.kind == GK_X) {
        for (int base = 0; base < D; ++base) {
            if ((base & tm) != 0 || (base & cm) != cm) continue;
            double *a = m + (size_t)base * row, *b = m + (size_t)(base | tm) * row;
            for (size_t i = 0; i < row; ++i) std::swap(a[i], b[i]);
        }
        return;
    }
    if (g.diag) {
        for (int base = 0; base < D; ++base) {
            if ((base & tm) != 0 || (base & cm) != cm) continue;
            for (int r = 0; r < T; ++r) {
                const double zr = g.m[(size_t)r * T + r].real(), zi = g.m[(size_t)r * T + r].imag();
                double *a = m + (size_t)(base | spread[r]) * row;
                for (int col = 0; col < D; ++col) {
                    const double xr = a[2 * col], xi = a[2 * col + 1];
                    a[2 * col] = zr * xr - zi * xi;
                    a[2 * col + 1] = zr * xi + zi * xr;
                }
            }
        }
        return;
    }
    std::vector<double> in((size_t)T * row);
    for (int base = 0; base < D; ++base) {
        if ((base & tm) != 0 || (base & cm) != cm) continue;
        for (int c = 0; c < T; ++c)
            std::copy_n(m + (size_t)(base | spread[c]) * row, row, in.data() + (size_t)c * row);
        for (int r = 0; r < T; ++r) {
            double *out = m + (size_t)(base | spread[r]) * row;
            std::fill_n(out, row, 0.0);
            for (int c = 0; c < T; ++c) {
                const double gr = g.m[(size_t)r * T + c].real(), gi = g.m[(size_t)r * T + c].imag();
                if (gr == 0.0 && gi == 0.0) continue;
                const double *x = in.data() + (size_t)c * row;
                for (int col = 0; col < D; ++col) {
                    out[2 * col] += gr * x[2 * col] - gi * x[2 * col + 1];
                    out[2 * col + 1] += gr * x[2 * col + 1] + gi * x[2 * col];
                }
            }
        }
    }
}

inline uint64_t qmask(const GateRec &g) { return g.tmask | g.cmask; }

}  // namespace

// Fraction of the amplitudes a plain launch of g reads and writes.
double touched_fraction(const GateRec &g) {
    int fixed = (int)g.controls.size() + (g.kind == GK_PHASE ? 1 : 0);
    return std::ldexp(1.0, -fixed);
}

// Table of a diagonal block over qubit set dmask: d[r] = product over the
// member gates of their diagonal entry for the assignment r of dmask (bit j
// of r = j-th lowest qubit of dmask); gates whose controls are not all 1
// in r contribute 1.
std::vector<cd> diag_table(const std::vector<GateRec> &q, const std::vector<int> &members, uint64_t dmask) {
    int pos[64], k = 0;
    for (int b = 0; b < 64; ++b) pos[b] = ((dmask >> b) & 1ull) ? k++ : -1;
    std::vector<cd> d((size_t)1 << k, cd(1.0, 0.0));
    for (int gi : members) {
        const GateRec &g = q[gi];
        const int T = 1 << g.t;
        for (size_t r = 0; r < d.size(); ++r) {
            bool on = true;
            for (int c : g.controls) on = on && ((r >> pos[c]) & 1u);
            if (!on) continue;
            int ti = 0;
            for (int j = 0; j < g.t; ++j) ti |= (int)((r >> pos[g.targets[j]]) & 1u) << j;
            d[r] *= g.m[(size_t)ti * T + ti];
        }
    }
    return d;
}

// f of a permutation block over qubit set pmask: each register value v
// (bit j = j-th lowest qubit of pmask) taken through the member gates in
// order (a gate whose controls are all 1 maps its target value c to
// pmap[c]).
std::vector<uint64_t> perm_table(const std::vector<GateRec> &q, const std::vector<int> &members, uint64_t pmask) {
    int pos[64], k = 0;
    for (int b = 0; b < 64; ++b) pos[b] = ((pmask >> b) & 1ull) ? k++ : -1;
    std::vector<uint64_t> f((size_t)1 << k);
    for (size_t v = 0; v < f.size(); ++v) {
        uint64_t x = v;
        for (int gi : members) {
            const GateRec &g = q[gi];
            bool on = true;
            for (int c : g.controls) on = on && ((x >> pos[c]) & 1u);
            if (!on) continue;
            unsigned c = 0;
            for (int j = 0; j < g.t; ++j) c |= (unsigned)((x >> pos[g.targets[j]]) & 1u) << j;
            const unsigned r = g.pmap[c];
            for (int j = 0; j < g.t; ++j) x = (x & ~(1ull << pos[g.targets[j]])) | ((uint64_t)((r >> j) & 1u) << pos[g.targets[j]]);
        }
        f[v] = x;
    }
    return f;
}

void block_matrix(const std::vector<GateRec> &q, PlanItem &it) {
    const auto t0 = std::chrono::steady_clock::now();
    if (it.diag_block) {
        it.dtab = diag_table(q, it.members, it.dmask);
    } else if (it.prod_block) {
        // per wire (ascending) the ordered product of its one-qubit gates
        std::vector<int> col(64, -1);
        int k = 0;
        for (int b = 0; b < 64; ++b)
            if ((it.qmask_prod >> b) & 1ull) col[b] = k++;
        it.pm.assign((size_t)4 * k, cd(0.0, 0.0));
        for (int j = 0; j < k; ++j) it.pm[4 * j] = it.pm[4 * j + 3] = 1.0;
        for (int gi : it.members) {
            const GateRec &g = q[gi];
            if (col[g.targets[0]] < 0) continue;  // a wire whose product is the identity
            cd *M = &it.pm[4 * (size_t)col[g.targets[0]]];
            const cd a = M[0], b = M[1], c = M[2], d = M[3];
            M[0] = g.m[0] * a + g.m[1] * c;
            M[1] = g.m[0] * b + g.m[1] * d;
            M[2] = g.m[2] * a + g.m[3] * c;
            M[3] = g.m[2] * b + g.m[3] * d;
        }
    } else if (it.perm_block) {
        it.ptab = perm_table(q, it.members, it.pmask);
    } else {
        const int D = 1 << it.k;
        it.m.assign((size_t)D * D, cd(0.0, 0.0));
        for (int i = 0; i < D; ++i) it.m[(size_t)i * D + i] = 1.0;
        for (int gi : it.members) apply_to_block(it.m, it.k, it.qubits, q[gi]);
    }
    it.host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

int perm_min_width(int prec, int kmax) { return prec == QSIM_C128 ? 1 : kmax + 1; }

bool butterfly2(const cd *u) {
    const double c = std::abs(u[0]);
    if (!(c > 0.0) || !std::isfinite(c)) return false;
    for (int e = 0; e < 4; ++e)
        if (std::abs(u[e].imag()) > 1e-12 * c || std::abs(std::abs(u[e].real()) - c) > 1e-12 * c) return false;
    const double s = (u[0].real() > 0) == (u[3].real() > 0) ? 1.0 : -1.0;  // s00 s11
    const double t = (u[1].real() > 0) == (u[2].real() > 0) ? 1.0 : -1.0;  // s01 s10
    return s == -t;
}

bool perm_map(const GateRec &g, std::vector<uint8_t> &pmap) {
    const int T = 1 << g.t;
    pmap.assign(T, 0);
    for (int c = 0; c < T; ++c) {
        int row = -1;
        for (int r = 0; r < T; ++r) {
            const cd z = g.m[(size_t)r * T + c];
            if (z == cd(1.0, 0.0)) {
                if (row >= 0) return false;
                row = r;
            } else if (z != cd(0.0, 0.0)) {
                return false;
            }
        }
        if (row < 0) return false;
        pmap[c] = (uint8_t)row;
    }
    std::vector<char> seen(T, 0);  // a column map onto distinct rows
    for (int c = 0; c < T; ++c) {
        if (seen[pmap[c]]) return false;
        seen[pmap[c]] = 1;
    }
    return true;
}

int plan_greedy_each(const std::vector<GateRec> &q, int n, int kmax, const std::function<int(PlanItem &)> &emit,
                     int diag_k, bool matrices, int perm_min, int prod_min, int tie) {
    const size_t G = q.size();
    if (G == 0) return 0;
    // per-wire gate lists in program order
    std::vector<std::vector<int>> wire(n);
    for (size_t i = 0; i < G; ++i)
        for (int b = 0; b < n; ++b)
            if ((qmask(q[i]) >> b) & 1ull) wire[b].push_back((int)i);
    std::vector<size_t> front(n, 0);  // position in wire[b] of the next gate
    std::vector<char> done(G, 0);
    std::vector<int> mark(G, 0);  // scratch of the look-ahead
    // Pending diagonal gates a diagonal block on the qubits S could absorb:
    // those whose earlier gates on every wire are all diagonal gates within
    // S, counted by walking each wire of S from its front
    std::vector<int> seen;
    auto reach = [&](uint64_t S) {
        int c = 0;
        seen.clear();
        for (int b = 0; b < n; ++b) {
            if (!((S >> b) & 1ull)) continue;
            for (size_t k = front[b]; k < wire[b].size(); ++k) {
                const int gi = wire[b][k];
                if (!q[gi].diag || (qmask(q[gi]) & ~S)) break;
                if (++mark[gi] == __builtin_popcountll(qmask(q[gi]))) ++c;
                seen.push_back(gi);
            }
        }
        for (int gi : seen) mark[gi] = 0;
        return c;
    };
    size_t remaining = G, next_seed = 0;

    auto is_ready = [&](int gi) {
        const uint64_t m = qmask(q[gi]);
        for (int b = 0; b < n; ++b)
            if ((m >> b) & 1ull) {
                if (front[b] >= wire[b].size() || wire[b][front[b]] != gi) return false;
            }
        return true;
    };
    auto take = [&](int gi) {
        done[gi] = 1;
        --remaining;
        const uint64_t m = qmask(q[gi]);
        for (int b = 0; b < n; ++b)
            if ((m >> b) & 1ull) ++front[b];
    };
    auto popc = [](uint64_t x) { return __builtin_popcountll(x); };
    auto untake = [&](int gi) {
        done[gi] = 0;
        ++remaining;
        const uint64_t m = qmask(q[gi]);
        for (int b = 0; b < n; ++b)
            if ((m >> b) & 1ull) --front[b];
    };

    while (remaining) {
        while (next_seed < G && done[next_seed]) ++next_seed;
        const int seed = (int)next_seed;  // earliest undone gate is always ready
        if (perm_min > 0 && q[seed].perm && popc(qmask(q[seed])) <= kMaxPermQubits) {
            // a permutation block: grow through the ready permutation gates
            // (fewest new qubits first, program order kept on every wire) up
            // to kMaxPermQubits qubits
            std::vector<int> pm;
            uint64_t Sp = qmask(q[seed]);
            double frac = touched_fraction(q[seed]);
            take(seed);
            pm.push_back(seed);
            for (;;) {
                int best = -1, best_add = 1 << 30;
                for (int b = 0; b < n; ++b) {
                    if (front[b] >= wire[b].size()) continue;
                    const int gi = wire[b][front[b]];
                    if (!q[gi].perm) continue;
                    const uint64_t m = qmask(q[gi]);
                    const int add = popc(m & ~Sp);
                    if (popc(Sp | m) > kMaxPermQubits || !is_ready(gi)) continue;
                    if (add < best_add || (add == best_add && gi < best)) {
                        best = gi;
                        best_add = add;
                    }
                }
                if (best < 0) break;
                take(best);
                pm.push_back(best);
                Sp |= qmask(q[best]);
                frac += touched_fraction(q[best]);
            }
            // its own pass only if wide enough (perm_min), cheaper than the
            // separate launches, and at least two gate incidences per qubit:
            // a single layer of permutation gates (the CNOTs of a brickwork
            // layer) rides along in the dense blocks that hold its
            // neighbours at no cost, and taking it out splits them (69 ->
            // 181 passes for a 32-qubit depth-40 brickwork); chains of
            // dependent permutation gates (adders, comparators) do not
            int incid = 0;
            for (int gi : pm) incid += popc(qmask(q[gi]));
            if (pm.size() >= 2 && frac >= 1.0 && popc(Sp) >= perm_min && incid >= 2 * popc(Sp)) {
                PlanItem it;
                it.fused = true;
                it.perm_block = true;
                it.pmask = Sp;
                it.k = popc(Sp);
                it.ngates = (int)pm.size();
                it.members = pm;
                for (int gi : pm) it.amp_updates += (double)(1ull << (n - (int)q[gi].controls.size()));
                if (matrices) block_matrix(q, it);
                if (const int rc = emit(it)) return rc;
                continue;
            }
            for (auto r = pm.rbegin(); r != pm.rend(); ++r) untake(*r);
        }
        if (diag_k > 0 && q[seed].diag && popc(qmask(q[seed])) <= diag_k) {
            // a diagonal block: ready diagonal gates commute with each other,
            // so absorb them (fewest new qubits first) up to diag_k qubits.
            // Among gates adding the same number of qubits, take the one
            // after which the block's qubits can absorb the most pending
            // diagonal gates: those whose earlier gates on every wire are all
            // diagonal gates on the block's qubits (a QFT's phase gates from
            // one group of qubits onto the next: about 36 per 12-qubit block,
            // where the earliest-first choice chains one control's gates onto
            // 11 new qubits)
            std::vector<int> dm;
            uint64_t Sd = qmask(q[seed]);
            double frac = touched_fraction(q[seed]);
            take(seed);
            dm.push_back(seed);
            for (;;) {
                int best = -1, best_add = 1 << 30, best_gain = -1;
                for (int b = 0; b < n; ++b) {
                    if (front[b] >= wire[b].size()) continue;
                    const int gi = wire[b][front[b]];
                    if (!q[gi].diag) continue;
                    const uint64_t m = qmask(q[gi]);
                    const int add = popc(m & ~Sd);
                    if (popc(Sd | m) > diag_k || !is_ready(gi)) continue;
                    if (add > best_add) continue;
                    const int gain = add > 0 ? reach(Sd | m) : 0;
                    if (add < best_add || gain > best_gain || (gain == best_gain && gi < best)) {
                        best = gi;
                        best_add = add;
                        best_gain = gain;
                    }
                }
                if (best < 0) break;
                take(best);
                dm.push_back(best);
                Sd |= qmask(q[best]);
                frac += touched_fraction(q[best]);
            }
            // worth one full pass only if the separate launches would touch more
            if (dm.size() >= 2 && frac >= 1.0) {
                PlanItem it;
                it.fused = true;
                it.diag_block = true;
                it.dmask = Sd;
                it.k = popc(Sd);
                it.ngates = (int)dm.size();
                it.members = dm;
                for (int gi : dm) it.amp_updates += (double)(1ull << (n - (int)q[gi].controls.size()));
                if (matrices) block_matrix(q, it);
                if (const int rc = emit(it)) return rc;
                continue;
            }
            for (auto r = dm.rbegin(); r != dm.rend(); ++r) untake(*r);
        }
        auto one_qubit = [&](int gi) { return q[gi].t == 1 && q[gi].controls.empty(); };
        if (prod_min > 0 && one_qubit(seed)) {
            // a product item: every ready uncontrolled one-qubit gate, wire
            // by wire in program order, on the wires whose next gate is
            // wider than kmax (or that end); worth it on prod_min wires
            std::vector<int> pr;
            uint64_t P = 0;
            for (bool again = true; again;) {
                again = false;
                for (int b = 0; b < n; ++b)
                    while (front[b] < wire[b].size() && one_qubit(wire[b][front[b]])) {
                        const int gi = wire[b][front[b]];
                        take(gi);
                        pr.push_back(gi);
                        P |= 1ull << b;
                        again = true;
                    }
            }
            for (int b = 0; b < n; ++b) {
                if (!((P >> b) & 1ull) || front[b] >= wire[b].size()) continue;
                if (popc(qmask(q[wire[b][front[b]]])) > kmax) continue;
                // this wire continues into a gate a dense block can take: its
                // one-qubit gates stay for that block
                for (auto r = pr.rbegin(); r != pr.rend(); ++r)
                    if (q[*r].targets[0] == b) untake(*r);
                pr.erase(std::remove_if(pr.begin(), pr.end(), [&](int gi) { return q[gi].targets[0] == b; }),
                         pr.end());
                P &= ~(1ull << b);
            }
            if (popc(P) >= prod_min) {
                PlanItem it;
                it.fused = true;
                it.prod_block = true;
                it.qmask_prod = P;
                it.ngates = (int)pr.size();
                it.members = pr;
                it.amp_updates = (double)pr.size() * (double)(1ull << n);
                block_matrix(q, it);
                // the pass takes butterfly matrices only; identity wires drop out
                uint64_t keep = 0;
                bool ok = true;
                for (int b = 0, k = 0; b < n; ++b) {
                    if (!((P >> b) & 1ull)) continue;
                    const cd *M = &it.pm[4 * (size_t)k++];
                    const bool ident = std::abs(M[0] - 1.0) <= 1e-12 && std::abs(M[1]) <= 1e-12 &&
                                       std::abs(M[2]) <= 1e-12 && std::abs(M[3] - 1.0) <= 1e-12;
                    if (butterfly2(M))
                        keep |= 1ull << b;
                    else if (!ident)
                        ok = false;
                }
                if (ok && popc(keep) >= prod_min) {
                    if (keep != P) {
                        it.qmask_prod = keep;
                        block_matrix(q, it);
                    }
                    if (const int rc = emit(it)) return rc;
                    continue;
                }
            }
            for (auto r = pr.rbegin(); r != pr.rend(); ++r) untake(*r);
        }
        if (popc(qmask(q[seed])) > kmax) {
            PlanItem it;
            it.fused = false;
            it.gate = seed;
            it.amp_updates = (double)(1ull << (n - (int)q[seed].controls.size()));
            it.ngates = 1;
            it.members.push_back(seed);
            take(seed);
            if (const int rc = emit(it)) return rc;
            continue;
        }
        std::vector<int> members;
        uint64_t S = qmask(q[seed]);
        take(seed);
        members.push_back(seed);
        for (;;) {
            bool absorbed = false;
            // 1) ready gates already inside S (repeat until none)
            for (bool again = true; again;) {
                again = false;
                for (int b = 0; b < n; ++b) {
                    if (!((S >> b) & 1ull) || front[b] >= wire[b].size()) continue;
                    const int gi = wire[b][front[b]];
                    const uint64_t m = qmask(q[gi]);
                    if ((m & ~S) == 0 && is_ready(gi)) {
                        take(gi);
                        members.push_back(gi);
                        again = absorbed = true;
                    }
                }
            }
            // 2) grow by the ready gate adding the fewest new qubits; among
            // those the earliest (tie 0), or the one sharing the most qubits
            // with the block (tie 1: a chain gate across the block's edge
            // before a one-qubit gate on a new wire).  Neither is better
            // everywhere: the 32-qubit depth-40 brickwork takes 69 passes
            // with tie 0 and 83 with tie 1, the circuit of the paper's Fig. 7
            // 12 and 6 (the diagonal blocks' look-ahead applied here: 73 for
            // the brickwork)
            int best = -1, best_new = 1 << 30, best_ov = -1;
            for (int b = 0; b < n; ++b) {
                if (front[b] >= wire[b].size()) continue;
                const int gi = wire[b][front[b]];
                const uint64_t m = qmask(q[gi]);
                const int add = popc(m & ~S);
                if (add == 0 || popc(S | m) > kmax) continue;
                if (!is_ready(gi)) continue;
                const int ov = tie == 1 ? popc(m & S) : 0;
                if (add < best_new || (add == best_new && (ov > best_ov || (ov == best_ov && gi < best)))) {
                    best = gi;
                    best_new = add;
                    best_ov = ov;
                }
            }
            if (best < 0) {
                if (!absorbed) break;
                continue;
            }
            S |= qmask(q[best]);
            take(best);
            members.push_back(best);
        }
        PlanItem it;
        it.ngates = (int)members.size();
        it.members = members;
        for (int gi : members) it.amp_updates += (double)(1ull << (n - (int)q[gi].controls.size()));
        if (members.size() == 1) {
            it.fused = false;
            it.gate = members[0];
        } else {
            it.fused = true;
            it.k = 0;
            for (int b = 0; b < n; ++b)
                if ((S >> b) & 1ull) it.qubits[it.k++] = b;
            if (matrices) block_matrix(q, it);
        }
        if (const int rc = emit(it)) return rc;
    }
    return 0;
}

void plan_greedy(const std::vector<GateRec> &q, int n, int kmax, std::vector<PlanItem> &out, int diag_k,
                 bool matrices, int perm_min, int prod_min, int tie) {
    out.clear();
    plan_greedy_each(
        q, n, kmax,
        [&](PlanItem &it) {
            out.push_back(std::move(it));
            return 0;
        },
        diag_k, matrices, perm_min, prod_min, tie);
}

// ---------------------------------------------------------------------------
// learned planner
// ---------------------------------------------------------------------------
// Features (all scaled to O(1)):
//  0 n/32            1 bytes per amplitude/16   2 fused block        3 tensor cores (1), c128 double-float (0.5)
//  4 width/5         5 gates in item/32         6 plain dense gate   7 plain phase gate
//  8 diagonal gate or block                     9 X gate or permutation block
// 10 controls/8      11 log2(fraction touched)/8
// 12 lowest qubit/32 13 highest qubit/32       14 qubits below 5 /5  15 constant 1
void item_features(const PlanItem &it, const std::vector<GateRec> &q, int n, int prec, bool tc_enabled, bool df,
                   float *f) {
    for (int i = 0; i < kFeatures; ++i) f[i] = 0.f;
    f[0] = n / 32.f;
    f[1] = (prec == QSIM_C128 ? 16.f : 8.f) / 16.f;
    f[15] = 1.f;
    // the executor's arithmetic: 1 for complex64 tensor-core blocks (below),
    // 0.5 for complex128 in double-float arithmetic, 0 otherwise
    if (prec == QSIM_C128 && df) f[3] = 0.5f;
    uint64_t mask = 0;
    if (it.fused && it.diag_block) {
        f[2] = 1.f;
        f[4] = it.k / 5.f;
        f[5] = it.ngates / 32.f;
        f[8] = 1.f;
        mask = it.dmask;
    } else if (it.fused && it.prod_block) {
        f[2] = 1.f;
        f[4] = __builtin_popcountll(it.qmask_prod) / 5.f;
        f[5] = it.ngates / 32.f;
        mask = it.qmask_prod;
    } else if (it.fused && it.perm_block) {
        f[2] = 1.f;
        f[4] = it.k / 5.f;
        f[5] = it.ngates / 32.f;
        f[9] = 1.f;
        mask = it.pmask;
    } else if (it.fused) {
        f[2] = 1.f;
        if (prec == QSIM_C64 && it.k >= 4 && n >= 12 && tc_enabled) f[3] = 1.f;
        f[4] = it.k / 5.f;
        f[5] = it.ngates / 32.f;
        for (int j = 0; j < it.k; ++j) mask |= 1ull << it.qubits[j];
    } else {
        const GateRec &g = q[it.gate];
        f[4] = g.t / 5.f;
        f[5] = 1.f / 32.f;
        f[6 + (g.kind == GK_PHASE ? 1 : g.kind == GK_DIAG1 ? 2 : g.kind == GK_X ? 3 : 0)] = 1.f;
        const int c = (int)g.controls.size();
        f[10] = c / 8.f;
        const int fixed = c + (g.kind == GK_PHASE ? 1 : 0);
        f[11] = -(float)fixed / 8.f;
        mask = g.tmask | g.cmask;
    }
    int lo = 64, hi = -1, low5 = 0;
    for (int b = 0; b < 64; ++b)
        if ((mask >> b) & 1ull) {
            lo = b < lo ? b : lo;
            hi = b;
            if (b < 5) ++low5;
        }
    f[12] = (lo == 64 ? 0 : lo) / 32.f;
    f[13] = (hi < 0 ? 0 : hi) / 32.f;
    f[14] = low5 / 5.f;
}

float CostModel::predict(const float *x) const {
    const int H = hidden;  // <= kMaxHidden (checked when the model is loaded)
    const float *W1 = p.data(), *b1 = W1 + (size_t)H * kFeatures, *W2 = b1 + H, *b2 = W2 + (size_t)H * H,
                *w3 = b2 + H, *b3 = w3 + H;
    float h1[kMaxHidden], h2[kMaxHidden];
    for (int j = 0; j < H; ++j) {
        float a = b1[j];
        for (int i = 0; i < kFeatures; ++i) a += W1[(size_t)j * kFeatures + i] * x[i];
        h1[j] = a > 0.f ? a : 0.f;
    }
    for (int j = 0; j < H; ++j) {
        float a = b2[j];
        for (int i = 0; i < H; ++i) a += W2[(size_t)j * H + i] * h1[i];
        h2[j] = a > 0.f ? a : 0.f;
    }
    float y = b3[0];
    for (int i = 0; i < H; ++i) y += w3[i] * h2[i];
    return y;
}

PlanItem single_item(const std::vector<GateRec> &q, int n, int gi) {
    PlanItem it;
    it.fused = false;
    it.gate = gi;
    it.ngates = 1;
    it.members.push_back(gi);
    it.amp_updates = (double)(1ull << (n - (int)q[gi].controls.size()));
    return it;
}

void plan_mlp(const std::vector<GateRec> &q, int n, int prec, bool tc_enabled, bool df, bool perm_blocks,
              int kmax_limit, const CostModel &cm,
              MlpChoice &choice) {
    auto cost = [&](const PlanItem &it) {
        float f[kFeatures];
        item_features(it, q, n, prec, tc_enabled, df, f);
        return std::exp((double)cm.predict(f));
    };
    // every gate's cost as a plain launch, predicted once
    std::vector<double> single(q.size());
    double total_single = 0.0;
    for (size_t gi = 0; gi < q.size(); ++gi) {
        single[gi] = cost(single_item(q, n, (int)gi));
        total_single += single[gi];
    }
    choice.kmax = 1;
    choice.fuse.clear();
    choice.predicted_ms = total_single;
    for (int kmax = 2; kmax <= kmax_limit; ++kmax) {
        std::vector<PlanItem> blocks;
        plan_greedy(q, n, kmax, blocks, kMaxDiagQubits, false, perm_blocks ? perm_min_width(prec, kmax) : 0);
        std::vector<char> fuse(blocks.size(), 0);
        double total = 0.0;
        for (size_t i = 0; i < blocks.size(); ++i) {
            const PlanItem &b = blocks[i];
            double cs = 0.0;
            for (int gi : b.members) cs += single[gi];
            if (!b.fused) {
                total += cs;
                continue;
            }
            const double cf = cost(b);
            fuse[i] = cf <= cs;
            total += fuse[i] ? cf : cs;
        }
        if (total < choice.predicted_ms) {
            choice.predicted_ms = total;
            choice.kmax = kmax;
            choice.fuse.swap(fuse);
        }
    }
}
