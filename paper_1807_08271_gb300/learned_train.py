"""Train the learned initialiser on the GPU with the library's own kernels.

Data: seeded synthetic 640x480 pairs (GPU ray caster, object scenes, relative
poses with a rotation angle ~U(0, max_angle) deg and a translation ~U(0,
max_trans) m), each labelled by the plain method: the batched coarse-to-fine
Gauss-Newton alignment (4 levels, [5, 5, 5, 10] iterations) started at the
ground truth; the label is its converged pose as a scaled twist.  Inputs: the
pairs' 80x60 pyramid level.  Training: Adam on the Gaussian NLL with a cosine
learning-rate schedule.  Calibration: on held-out pairs, the largest
log-variance threshold under which the proposals stay inside a safe start
region (rotation and translation error bounds) for all but a small fraction.

    python -m paper_1807_08271_gb300.learned_train --pairs 200000 --out weights.npz
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import time

import numpy as np

from . import rgbid as R
from .batch import BatchAligner
from .learned import InitNet, twist_of_pose
from .synth import gpu as G

LEVELS, ITERS = 4, [5, 5, 5, 10]
CONV_ROT, CONV_TRANS = 2e-3, 5e-3        # "converged": within 2 mrad and 5 mm of the label


def label_chunk(seed: int, n: int, bank, precision: int, max_angle: float, max_trans: float):
    """Render n pairs, label them with the batched plain alignment started at the
    ground truth, and pack the network inputs.  Returns (x [n, 60, 80, 4] bf16,
    twist labels [n, 6] float64, ground truth [n, 4, 4], keep mask [n])."""
    import torch
    d = G.make_pairs_gpu(seed, n, bank, 640, 480, max_angle, max_trans)
    pyr, items = [], []
    for i in range(n):
        PA = R.DevicePyramid(640, 480, LEVELS, precision).build(d["I"][i, 0], d["W"][i, 0], d["K"])
        PB = R.DevicePyramid(640, 480, LEVELS, precision).build(d["I"][i, 1], d["W"][i, 1], d["K"])
        pyr.append((PA, PB))
        items.append(dict(ref=PA.desc, cur=PB.desc, T_init=d["T_gt"][i], levels=LEVELS, iters=ITERS))
    B = BatchAligner(items, precision=precision)
    B.config = R.BatchConfig(8, 2, 0, 0)
    B.run()
    x_slots = torch.empty((n, R.NET_IN_H, R.NET_IN_W, R.NET_IN_C), dtype=torch.bfloat16, device=B.d_items.device)
    R.rgbid_net_inputs(B.d_items, n, precision, x_slots)
    torch.cuda.synchronize()
    x = torch.empty_like(x_slots)
    x[torch.tensor(B.order, device=x.device)] = x_slots          # slot s holds item B.order[s]
    res = B.all_results()
    labels = np.zeros((n, 6))
    keep = np.zeros(n, dtype=bool)
    for i, r in enumerate(res):
        labels[i] = twist_of_pose(r["T"])
        E = np.linalg.inv(r["T"]) @ d["T_gt"][i]
        rot = math.acos(max(-1.0, min(1.0, (np.trace(E[:3, :3]) - 1) / 2)))
        keep[i] = r["status"] == R.OK and rot < math.radians(2.0) and np.linalg.norm(E[:3, 3]) < 0.05
    del pyr
    return x, labels, d["T_gt"], keep


def build_dataset(seed: int, n: int, bank, precision: int, max_angle: float, max_trans: float, chunk: int, log):
    import torch
    xs, ys, ts = [], [], []
    t0 = time.time()
    for c in range((n + chunk - 1) // chunk):
        m = min(chunk, n - c * chunk)
        x, lab, tgt, keep = label_chunk(seed * 1000003 + c, m, bank, precision, max_angle, max_trans)
        k = torch.from_numpy(np.nonzero(keep)[0]).to(x.device)
        xs.append(x[k])
        ys.append(torch.from_numpy((lab[keep] / R.NET_TWIST_SCALE).astype(np.float32)).to(x.device))
        ts.append(tgt[keep])
        log(f"chunk {c}: {m} pairs, kept {int(keep.sum())}, {time.time() - t0:.1f} s")
    return torch.cat(xs), torch.cat(ys), np.concatenate(ts)


def augment(xb, yb, gen):
    """Label-consistent augmentation of a batch (torch ops on the device):
    swap A and B (the twist of the inverse pose), mirror both frames left-right
    (t -> (-tx, ty, tz), w -> (wx, -wy, -wz)) and up-down (t -> (tx, -ty, tz),
    w -> (-wx, wy, -wz)); the 80x60 level's principal point is the image centre,
    so mirroring keeps the intrinsics.  Each sample gets each transform with
    probability 1/2."""
    import torch
    n = xb.shape[0]
    r = torch.rand((n, 3), generator=gen, device=xb.device) < 0.5
    x, y = xb.clone(), yb.clone()
    s = r[:, 0]
    if bool(s.any()):
        # inverse of the decoupled pose: R' = R^T, t' = -R^T t, w' = -w
        tw = y[s].double() * R.NET_TWIST_SCALE
        w = tw[:, 3:]
        th = torch.linalg.norm(w, dim=1, keepdim=True).clamp_min(1e-12)
        k = w / th
        K = torch.zeros((w.shape[0], 3, 3), dtype=torch.float64, device=x.device)
        K[:, 0, 1], K[:, 0, 2], K[:, 1, 2] = -k[:, 2], k[:, 1], -k[:, 0]
        K = K - K.transpose(1, 2)
        st, ct = torch.sin(th)[:, :, None], torch.cos(th)[:, :, None]
        Rm = torch.eye(3, dtype=torch.float64, device=x.device) + st * K + (1 - ct) * (K @ K)
        t_new = -(Rm.transpose(1, 2) @ tw[:, :3, None])[:, :, 0]
        y[s] = (torch.cat([t_new, -w], dim=1) / R.NET_TWIST_SCALE).float()
        x[s] = x[s][..., [2, 3, 0, 1]]
    h = r[:, 1]
    if bool(h.any()):
        x[h] = torch.flip(x[h], dims=[2])
        y[h] = y[h] * torch.tensor([-1.0, 1.0, 1.0, 1.0, -1.0, -1.0], device=y.device)
    v = r[:, 2]
    if bool(v.any()):
        x[v] = torch.flip(x[v], dims=[1])
        y[v] = y[v] * torch.tensor([1.0, -1.0, 1.0, -1.0, 1.0, -1.0], device=y.device)
    return x.contiguous(), y.contiguous()


def train(net: InitNet, X, Y, epochs: int, batch: int, lr: float, seed: int, log, augmented: bool = True):
    import torch
    n = X.shape[0]
    gen = torch.Generator(device=X.device)
    gen.manual_seed(seed)
    steps = epochs * (n // batch)
    warm = max(1, steps // 50)
    hist = []
    s = 0
    t0 = time.time()
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen, device=X.device)
        acc = torch.zeros((), device=X.device)
        nb = n // batch
        for b in range(nb):
            idx = perm[b * batch:(b + 1) * batch]
            xb = X.index_select(0, idx).contiguous()
            yb = Y.index_select(0, idx).contiguous()
            if augmented:
                xb, yb = augment(xb, yb, gen)
            rate = lr * min(1.0, (s + 1) / warm) * 0.5 * (1.0 + math.cos(math.pi * s / steps))
            acc += net.train_step(xb, yb, batch, rate)[0]
            s += 1
        mean = float(acc) / nb
        hist.append(mean)
        log(f"epoch {ep}: mean loss {mean:.4f} ({time.time() - t0:.1f} s)")
    return hist


def predict(net: InitNet, X):
    import torch
    out = []
    for b in range(0, X.shape[0], net.max_batch):
        xb = X[b:b + net.max_batch].contiguous()
        out.append(net.forward(xb, xb.shape[0]).clone())
    torch.cuda.synchronize()
    return torch.cat(out).cpu().numpy().astype(np.float64)


def proposal_errors(y, labels_scaled):
    """Rotation (rad) and translation (m) error of each proposal against its label."""
    d = (y[:, :6] - labels_scaled) * R.NET_TWIST_SCALE
    return np.linalg.norm(d[:, 3:], axis=1), np.linalg.norm(d[:, :3], axis=1)


def calibrate(y, labels_scaled, rot_bound: float, trans_bound: float, miss: float):
    """Largest log-variance threshold whose accepted proposals exceed the bounds for
    at most a fraction `miss` of them."""
    er, et = proposal_errors(y, labels_scaled)
    bad = (er > rot_bound) | (et > trans_bound)
    s = y[:, 6]
    order = np.argsort(s)
    cum_bad = np.cumsum(bad[order])
    best = -1e9
    for k in range(len(order)):
        if cum_bad[k] <= miss * (k + 1):
            best = s[order[k]]
    return float(best), float(np.mean(s <= best))


def _rot_angle(E) -> float:
    return math.acos(max(-1.0, min(1.0, (np.trace(np.asarray(E)[:3, :3]) - 1.0) / 2.0)))


def pose_diff(A, B):
    """(rotation angle rad, translation m) of A^-1 B."""
    E = np.linalg.inv(A) @ B
    return _rot_angle(E), float(np.linalg.norm(E[:3, 3]))


class EvalSet:
    """Held-out 640x480 pairs with their pyramids, batch items (identity start)
    and the plain method's converged pose from the ground truth (the label)."""

    def __init__(self, seed: int, n: int, bank, max_angle: float, max_trans: float):
        d = G.make_pairs_gpu(seed, n, bank, 640, 480, max_angle, max_trans)
        self.n, self.T_gt, self.pyr, self.items = n, d["T_gt"], [], []
        for i in range(n):
            PA = R.DevicePyramid(640, 480, LEVELS).build(d["I"][i, 0], d["W"][i, 0], d["K"])
            PB = R.DevicePyramid(640, 480, LEVELS).build(d["I"][i, 1], d["W"][i, 1], d["K"])
            self.pyr.append((PA, PB))
            self.items.append(dict(ref=PA.desc, cur=PB.desc, T_init=None, levels=LEVELS, iters=ITERS))
        lab = BatchAligner([dict(it, T_init=self.T_gt[i]) for i, it in enumerate(self.items)])
        lab.config = R.BatchConfig(8, 2, 0, 0)
        lab.run()
        self.labels = [r["T"] for r in lab.all_results()]

    def run(self, planner_factory=None, reps: int = 0):
        """Align the set in one batched launch; returns (results, ms per batch or None, aligner)."""
        import torch
        B = BatchAligner(self.items, planner_factory=planner_factory)
        if reps:
            B.tune(reps=2)
            B.capture()
            B.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                B.replay()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
        else:
            B.config = R.BatchConfig(8, 2, 0, 0)
            B.run()
            ms = None
        return B.all_results(), ms, B

    def converged(self, results, rot_tol: float = CONV_ROT, trans_tol: float = CONV_TRANS):
        """Per pair: does the final pose lie within (rot_tol rad, trans_tol m) of the
        label, i.e. in the basin the plain method converges to from the truth?"""
        out = []
        for r, L in zip(results, self.labels):
            dr, dt = pose_diff(r["T"], L)
            out.append(dr <= rot_tol and dt <= trans_tol)
        return np.array(out)


def calibrate_tiers(net: InitNet, cal: EvalSet, max_tier: int = 2):
    """Thresholds of tiers 1..max_tier.  For tier k the calibration set is aligned
    from every proposal with k coarse levels skipped; the threshold is the
    predicted log-variance of the largest most-confident prefix of pairs on which
    this converges at least as often as the plain alignment (identity start, all
    levels) on the same pairs, with a median distance to the label no larger
    than the plain alignment's (5 % slack).  Returns (thresholds, report)."""
    from .learned import LearnedPlanner
    res_p, _, _ = cal.run(None)
    ok_p = cal.converged(res_p)
    err_p = np.array([pose_diff(r["T"], L)[0] for r, L in zip(res_p, cal.labels)])
    thresholds, report = [], {"plain_converged": float(np.mean(ok_p))}
    for k in range(1, max_tier + 1):
        res, _, B = cal.run(lambda m, prec: LearnedPlanner(_sized(net, m), m, prec, [1e30] * k))
        ok = cal.converged(res)
        err = np.array([pose_diff(r["T"], L)[0] for r, L in zip(res, cal.labels)])
        y = B.planner.net.y[:cal.n, 6].cpu().numpy()
        s = np.zeros(cal.n)
        for slot in range(cal.n):
            s[B.order[slot]] = y[slot]
        order = np.argsort(s)
        cum_k, cum_p = np.cumsum(ok[order]), np.cumsum(ok_p[order])
        last = -1
        for j in range(cal.n):
            if cum_k[j] >= cum_p[j] and \
                    np.median(err[order[:j + 1]]) <= 1.05 * np.median(err_p[order[:j + 1]]) + 1e-7:
                last = j
        thr = float(s[order[last]]) + 1e-6 if last >= 0 else -1e30
        if thresholds:
            thr = min(thr, thresholds[-1])
        thresholds.append(thr)
        report[f"tier{k}"] = dict(threshold=thr, accepted=float(np.mean(s <= thr)),
                                  converged_all_confident=float(np.mean(ok)))
    return thresholds, report


def _sized(net: InitNet, n: int) -> InitNet:
    """The same parameters in a network whose workspace holds n inputs."""
    if n <= net.max_batch:
        return net
    big = InitNet(max_batch=n, device=net.device)
    big.params.copy_(net.params)
    return big


def evaluate_per_pair(net: InitNet, ev: EvalSet, thresholds, n: int) -> dict:
    """The first n pairs one at a time (rgbid_align per pair) from the identity
    with the plain schedule, and with the learned start (LearnedAligner): GPU time
    of the whole sequence of alignments, iterations and convergence."""
    import torch
    from .learned import LearnedAligner
    params = R.rgbid_default_params(levels=LEVELS, iters=ITERS)
    ws = R.new_workspace(ev.pyr[0][0].desc, params)
    res = R.result_tensor(n)
    la = LearnedAligner(_sized(net, 1), thresholds, levels=LEVELS, iters=ITERS)
    la.set_pairs([(ev.pyr[i][0].desc, ev.pyr[i][1].desc) for i in range(n)])
    out = {}
    for name in ("plain", "learned"):
        def one(i):
            PA, PB = ev.pyr[i]
            if name == "plain":
                R.rgbid_align(PA.desc, PB.desc, None, params, ws, res[i])
            else:
                la.align(i, ws, res[i])
        for i in range(min(n, 8)):
            one(i)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(n):
            one(i)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        rr = [R.parse_result(res[i]) for i in range(n)]
        ok = ev.converged(rr)
        out[name] = dict(alignments_per_s=n / (ms / 1e3), ms_per_alignment=ms / n,
                         mean_iterations=float(np.mean([r["iters_done"] for r in rr])),
                         converged_fraction=float(np.mean(ok)),
                         median_rot_err_vs_truth_rad=float(np.median([pose_diff(r["T"], T)[0]
                                                                      for r, T in zip(rr, ev.T_gt)])))
    # the network's share: the pair's item copied into place, then the inputs, forward
    # pass and plan (one graph replay in the aligner) of every pair alone
    size = ctypes.sizeof(R.BatchItem)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(n):
        la.d_one.copy_(la.d_src[i * size:(i + 1) * size], non_blocking=True)
        if la._graph is not None:
            la._graph.replay()
        else:
            la._plan()
    e1.record()
    torch.cuda.synchronize()
    out["network_ms_per_pair"] = e0.elapsed_time(e1) / n
    out["pairs"] = n
    return out


class _Ptr:
    def __init__(self, p):
        self.p = p

    def data_ptr(self):
        return self.p


def evaluate(net: InitNet, ev: EvalSet, thresholds, reps: int = 5, per_pair: int = 256) -> dict:
    """Plain form (identity start, all levels) against the learned form (proposal and
    skipped coarse levels where confident, plain otherwise) on held-out pairs:
    agreement with the plain method's converged pose, Gauss-Newton iterations and
    alignments/s, each form in one batched launch replayed from a CUDA graph."""
    from .learned import LearnedPlanner
    out, poses, agree = {}, {}, {}
    for name, factory in (("plain", None),
                          ("learned", lambda m, prec: LearnedPlanner(_sized(net, m), m, prec, thresholds))):
        res, ms, B = ev.run(factory, reps=reps)
        agree[name] = ev.converged(res)
        poses[name] = [r["T"] for r in res]
        out[name] = dict(ms_per_batch=ms, alignments_per_s=ev.n / (ms / 1e3),
                         mean_iterations=float(np.mean([r["iters_done"] for r in res])),
                         converged_fraction=float(np.mean(agree[name])),
                         median_rot_err_vs_truth_rad=float(np.median([pose_diff(r["T"], T)[0]
                                                                      for r, T in zip(res, ev.T_gt)])),
                         skipped_levels_histogram=(np.bincount(B.planner.skipped[:ev.n].cpu().numpy(),
                                                               minlength=3).tolist() if B.planner else None),
                         shape=list(B.config.as_tuple()))
    out["per_pair"] = evaluate_per_pair(net, ev, thresholds, min(ev.n, per_pair))
    d = [max(pose_diff(a, b)) for a, b, k in zip(poses["plain"], poses["learned"], agree["plain"]) if k]
    out["max_diff_learned_vs_plain_where_plain_converged"] = float(max(d)) if d else None
    out["median_diff_learned_vs_plain_where_plain_converged"] = float(np.median(d)) if d else None
    out["learned_converged_where_plain_converged"] = float(np.mean(agree["learned"][agree["plain"]]))
    out["pairs"] = ev.n
    return out


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=200000)
    ap.add_argument("--val", type=int, default=4096)
    ap.add_argument("--chunk", type=int, default=2048)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--max-angle", type=float, default=10.0)
    ap.add_argument("--max-trans", type=float, default=0.15)
    ap.add_argument("--cal-pairs", type=int, default=2048)
    ap.add_argument("--no-augment", action="store_true")
    ap.add_argument("--eval-pairs", type=int, default=256)
    ap.add_argument("--from-weights", default=None,
                    help="skip the training set and training: calibrate and evaluate these weights")
    ap.add_argument("--out", required=True)
    ap.add_argument("--log", default=None)
    a = ap.parse_args(argv)
    lines = []

    def log(msg):
        print(msg, flush=True)
        lines.append(msg)

    torch.cuda.set_device(0)
    bank = G.TextureBank(a.seed, device="cuda")
    if a.from_weights:
        net = InitNet.load(a.from_weights, max_batch=a.batch)
        for stale in ("max_log_var", "skip_levels", "accepted_on_calibration", "evaluation", "thresholds",
                      "calibration"):
            net.meta.pop(stale, None)
        hist = net.meta.get("loss_per_epoch", [])
        stats = {k: v for k, v in net.meta.items() if k.startswith("val_")}
        X = np.zeros((net.meta.get("train_pairs", 0), 1))
    else:
        X, Y, _ = build_dataset(a.seed, a.pairs, bank, R.PLANES_F32, a.max_angle, a.max_trans, a.chunk, log)
        Xv, Yv, _ = build_dataset(a.seed + 7919, a.val, bank, R.PLANES_F32, a.max_angle, a.max_trans, a.chunk, log)
        log(f"dataset: {X.shape[0]} training, {Xv.shape[0]} held-out pairs")
        net = InitNet(max_batch=a.batch, seed=a.seed)
        hist = train(net, X, Y, a.epochs, a.batch, a.lr, a.seed, log, augmented=not a.no_augment)
        yv = predict(net, Xv)
        lv = Yv.cpu().numpy().astype(np.float64)
        er, et = proposal_errors(yv, lv)
        stats = dict(val_rot_err_median_deg=float(np.degrees(np.median(er))),
                     val_rot_err_p95_deg=float(np.degrees(np.percentile(er, 95))),
                     val_trans_err_median_m=float(np.median(et)), val_trans_err_p95_m=float(np.percentile(et, 95)))
        log(json.dumps(stats))
    cal = EvalSet(a.seed + 7, a.cal_pairs, bank, a.max_angle, a.max_trans)
    thresholds, rep = calibrate_tiers(net, cal)
    log(json.dumps(dict(calibration=rep)))
    if a.from_weights:
        net.save(a.out, thresholds=thresholds, calibration=rep)
    else:
        net.save(a.out, thresholds=thresholds, calibration=rep, train_pairs=int(X.shape[0]), epochs=a.epochs,
                 batch=a.batch, lr=a.lr, seed=a.seed, max_angle_deg=a.max_angle, max_trans_m=a.max_trans,
                 loss_per_epoch=hist, **stats)
    if a.eval_pairs > 0:
        evals = {}
        for tag, ma, mt in (("train_range", a.max_angle, a.max_trans), ("half_range", a.max_angle / 2, a.max_trans / 2)):
            ev = EvalSet(a.seed + 104729, a.eval_pairs, bank, ma, mt)
            evals[tag] = evaluate(net, ev, thresholds)
            log(json.dumps({tag: evals[tag]}))
        net.save(a.out, evaluation=evals)
    if a.log:
        with open(a.log, "w") as f:
            f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
