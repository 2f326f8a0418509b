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
// FP64.  Gates on more than kmax qubits (e.g. a many-controlled Z) run alone
// with their specialised plain kernel.
#include <algorithm>
#include <cstring>

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
        out.push_back(std::move(it));
    }
}

namespace {

// Apply gate g to every column of the 2^k x 2^k matrix M (column-major view
// of a k-qubit register whose bit j is qubit S[j]):  M <- G M.
void apply_to_block(std::vector<cd> &M, int k, const int *S, const GateRec &g) {
    const int D = 1 << k;
    auto pos = [&](int qubit) {
        for (int j = 0; j < k; ++j)
            if (S[j] == qubit) return j;
        return -1;
    };
    int tpos[5];
    for (int j = 0; j < g.t; ++j) tpos[j] = pos(g.targets[j]);
    int cm = 0;
    for (int c : g.controls) cm |= 1 << pos(c);
    int tm = 0;
    for (int j = 0; j < g.t; ++j) tm |= 1 << tpos[j];
    const int T = 1 << g.t;
    std::vector<cd> in(T), outv(T);
    std::vector<int> idx(T);
    for (int col = 0; col < D; ++col) {
        for (int base = 0; base < D; ++base) {
            if ((base & tm) != 0 || (base & cm) != cm) continue;
            for (int r = 0; r < T; ++r) {
                int i = base;
                for (int j = 0; j < g.t; ++j)
                    if ((r >> j) & 1) i |= 1 << tpos[j];
                idx[r] = i;
                in[r] = M[(size_t)i * D + col];
            }
            for (int r = 0; r < T; ++r) {
                cd acc = 0;
                for (int c = 0; c < T; ++c) acc += g.m[(size_t)r * T + c] * in[c];
                outv[r] = acc;
            }
            for (int r = 0; r < T; ++r) M[(size_t)idx[r] * D + col] = outv[r];
        }
    }
}

inline uint64_t qmask(const GateRec &g) { return g.tmask | g.cmask; }

}  // namespace

void plan_greedy(const std::vector<GateRec> &q, int n, int kmax, std::vector<PlanItem> &out) {
    out.clear();
    const size_t G = q.size();
    if (G == 0) return;
    // per-wire gate lists in program order
    std::vector<std::vector<int>> wire(n);
    for (size_t i = 0; i < G; ++i)
        for (int b = 0; b < n; ++b)
            if ((qmask(q[i]) >> b) & 1ull) wire[b].push_back((int)i);
    std::vector<size_t> front(n, 0);  // position in wire[b] of the next gate
    std::vector<char> done(G, 0);
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

    while (remaining) {
        while (next_seed < G && done[next_seed]) ++next_seed;
        const int seed = (int)next_seed;  // earliest undone gate is always ready
        if (popc(qmask(q[seed])) > kmax) {
            PlanItem it;
            it.fused = false;
            it.gate = seed;
            it.amp_updates = (double)(1ull << (n - (int)q[seed].controls.size()));
            it.ngates = 1;
            take(seed);
            out.push_back(std::move(it));
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
            // 2) grow by the ready gate adding the fewest new qubits
            int best = -1, best_new = 1 << 30;
            for (int b = 0; b < n; ++b) {
                if (front[b] >= wire[b].size()) continue;
                const int gi = wire[b][front[b]];
                const uint64_t m = qmask(q[gi]);
                const int add = popc(m & ~S);
                if (add == 0 || popc(S | m) > kmax) continue;
                if (!is_ready(gi)) continue;
                if (add < best_new || (add == best_new && gi < best)) {
                    best = gi;
                    best_new = add;
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
        for (int gi : members) it.amp_updates += (double)(1ull << (n - (int)q[gi].controls.size()));
        if (members.size() == 1) {
            it.fused = false;
            it.gate = members[0];
        } else {
            it.fused = true;
            it.k = 0;
            for (int b = 0; b < n; ++b)
                if ((S >> b) & 1ull) it.qubits[it.k++] = b;
            const int D = 1 << it.k;
            it.m.assign((size_t)D * D, cd(0.0, 0.0));
            for (int i = 0; i < D; ++i) it.m[(size_t)i * D + i] = 1.0;
            for (int gi : members) apply_to_block(it.m, it.k, it.qubits, q[gi]);
        }
        out.push_back(std::move(it));
    }
}
