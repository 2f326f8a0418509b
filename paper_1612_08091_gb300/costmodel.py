"""Training data, training and storage of the learned planner's cost model.

The simulator times its own launches (profiling mode 2 records the 16
features of each planned item and its CUDA-event duration); the network is
trained on the GPU by the library's MLP kernels to predict log(ms); the
weights are loaded into a handle with ``Simulator.set_cost_model`` and used
by fusion mode "mlp".
"""
import json
import math
import os

import numpy as np

import circuitgen as cg

from .qsim import MLP, Simulator

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_MODEL = os.path.join(HERE, "data", "costmodel.json")


def training_circuits(n, seed):
    """The circuit families the model is trained on: random brickwork, QFT on
    a basis state, and the H / controlled-RZ chain / H circuit."""
    x = cg.random_basis_state(n, seed)
    return {
        "random": cg.random_u3_brickwork(n, 4, seed),
        "qft": cg.basis_prep_ops(x, n) + cg.qft_ops(n),
        "hcrz": cg.hadamard_crz_chain(n, seed),
    }


def collect(sizes=(26, 27, 28), precisions=("c64", "c128"), kmaxes=(1, 2, 3, 4, 5, 6), seed=2018, repeats=1,
            df=False):
    """Run every training circuit under every plan width and return the
    per-launch features (N x 16) and durations in ms (N).  Width 6 exists
    only for complex64 (tensor cores), so complex128 skips it.  df: complex128
    handles compute in double-float arithmetic."""
    feats, ms = [], []
    for n in sizes:
        circuits = training_circuits(n, seed + n)
        for prec in precisions:
            for kmax in kmaxes:
                if kmax > 5 and prec != "c64":
                    continue
                fusion = "none" if kmax == 1 else "greedy"
                with Simulator(n, precision=prec, fusion=fusion, kmax=max(kmax, 1), c128_df=df) as sim:
                    for _ in range(repeats + 1):
                        for ops in circuits.values():
                            sim.reset(0)
                            sim.set_profiling(2)
                            sim.run(ops)
                            sim.flush()
                            f, t = sim.item_times()
                            feats.append(f)
                            ms.append(t)
    return np.concatenate(feats), np.concatenate(ms)


def train(X, ms, hidden=32, epochs=400, batch=256, lr=3e-3, seed=7):
    """Fit log(ms) with the GPU-trained MLP; returns (params, final loss)."""
    y = np.log(np.maximum(ms, 1e-4)).astype(np.float32)
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(y))
    net = MLP(hidden=hidden, seed=seed)
    loss = net.train(X[order], y[order], epochs=epochs, batch=batch, lr=lr)
    params = net.params
    net.close()
    return params, loss


def save(params, hidden, path=DEFAULT_MODEL, meta=None):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump({"hidden": int(hidden), "params": [float(v) for v in params], "meta": meta or {}}, f)


def load(path=DEFAULT_MODEL):
    with open(path) as f:
        d = json.load(f)
    return np.asarray(d["params"], dtype=np.float32), int(d["hidden"])


def main():
    import argparse

    ap = argparse.ArgumentParser(description="collect timings on this GPU, train the cost model, save it")
    ap.add_argument("--sizes", default="26,27,28")
    ap.add_argument("--hidden", type=int, default=32)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--out", default=DEFAULT_MODEL)
    a = ap.parse_args()
    sizes = tuple(int(v) for v in a.sizes.split(","))
    X, ms = collect(sizes=sizes)
    params, loss = train(X, ms, hidden=a.hidden, epochs=a.epochs)
    save(params, a.hidden, a.out, meta={"samples": int(len(ms)), "sizes": list(sizes), "train_mse_log": loss})
    print(json.dumps({"samples": int(len(ms)), "train_mse_log": loss, "rms_rel": math.sqrt(loss), "out": a.out}))


if __name__ == "__main__":
    main()
