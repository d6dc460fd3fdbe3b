"""Train the learned initial guess of step 1 on rows generated by the plain SSM.

Rows (features, converged pair sum) come from plain FP32C runs of the coupled
workload (d = 3, h = 2^-8, T = 1) over seeds 100..163: after every step each run
contributes an evenly strided sample of its particles (offset rotating with the
step).  The network is then trained on the GPU by the library's own kernels
(ssm_ws_train) and the blob is written to --out.

  python -m paper_2105_09688_gb300.train_ws --N 65536 --rows 10000000 --epochs 20 \\
      --out paper_2105_09688_gb300/ws_weights.bin
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def generate(S, N, seeds, rows, h=2.0 ** -8, T=1.0):
    steps = int(round(T / h))
    per_step = max(1, rows // (len(seeds) * steps))
    stride = max(1, N // per_step)
    feats, labels = [], []
    for seed in seeds:
        s = S.SSM(d=3, N=N, h=h, T=T, coef=S.SSM_COEF_COUPLED3D, seed=seed, precision=S.SSM_FP32C)
        for n in range(steps):
            s.step()
            f, l = s.ws_collect(stride, n % stride)
            feats.append(f)
            labels.append(l)
        s.close()
    return np.concatenate(feats), np.concatenate(labels), stride


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=65536)
    ap.add_argument("--seed-first", type=int, default=100)
    ap.add_argument("--seed-count", type=int, default=64)
    ap.add_argument("--rows", type=int, default=10_000_000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default=os.path.join(HERE, "ws_weights.bin"))
    a = ap.parse_args()
    from paper_2105_09688_gb300 import build as B
    B.build()
    import paper_2105_09688_gb300 as S
    t0 = time.time()
    seeds = list(range(a.seed_first, a.seed_first + a.seed_count))
    feat, label, stride = generate(S, a.N, seeds, a.rows)
    t1 = time.time()
    blob, curve = S.ssm_ws_train(feat, label, epochs=a.epochs, batch=a.batch, lr=a.lr, seed=0)
    t2 = time.time()
    with open(a.out, "wb") as f:
        f.write(blob)
    print(json.dumps({"rows": int(feat.shape[0]), "N": a.N, "seeds": [seeds[0], seeds[-1]], "stride": stride,
                      "gen_s": t1 - t0, "train_s": t2 - t1, "loss_curve": [float(v) for v in curve],
                      "out": a.out}))


if __name__ == "__main__":
    main()
