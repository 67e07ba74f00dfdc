"""Training of the learned hole-repair network on pairs the method generates.

A pair is one stereo frame of a seeded synthetic scene: the features of the
affiliated eye after the forward warp (gs_repair_features), the full affiliated
render (gs_render_two_pass) as the target, and the interpolation-only
affiliated image (gs_render_stereo with the centre step off: gaps interpolated,
remaining holes filled along their row or column) as the plain fill the gate
compares against. Frames stay resident on the GPU; every step draws a random
set of 16x16 tiles that contain holes outside the edge strips (the tiles the
network serves at inference) and runs gs_repair_train_step (forward on the
tensor cores, FP32 gradients, AdamW) through the C ABI.

    python -m paper_2609_30741_gb300.repair_train --scene object --scenes 4 \\
        --poses 6 --steps 1500 --out weights.npy [--checkpoint ck.npz
        --checkpoint-every 100] [--resume ck.npz]

The packaged weights (UNBOUNDED_WEIGHTS) come from 2,000 pairs of the
unbounded distribution, 50 scenes (seeds 7000-7049, 1.5M surfels, 1920x1080)
x 40 random head poses, streamed in shards of 250 frames over two epochs:

    python -m paper_2609_30741_gb300.repair_train --scene unbounded --scenes 50 \\
        --poses 40 --shard 250 --epochs 2 --steps 150 --eval-scenes 2 \\
        --out paper_2609_30741_gb300/weights/repair_unbounded_2000pairs.npy
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import gs, synth

UNBOUNDED_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                                 "repair_unbounded_2000pairs.npy")
UNBOUNDED_TRAINING = {"pairs": 2000, "scenes": "unbounded seeds 7000-7049, 1.5M surfels, 1920x1080",
                      "poses_per_scene": 40, "shard_frames": 250, "epochs": 2, "steps": 2400,
                      "batch_tiles": 512}


def init_weights(seed: int, gate_bias: float = -2.0) -> np.ndarray:
    """He-normal weights and zero biases for the first five layers; the last
    layer starts at zero (the fill starts as the method's own fill) with a gate
    bias that keeps every tile on the plain path until training opens it."""
    rng = np.random.default_rng(seed)
    chans = (6, 32, 32, 32, 32, 32, 4)
    parts = []
    for l in range(6):
        ci, co = chans[l], chans[l + 1]
        if l < 5:
            parts.append(rng.normal(0.0, math.sqrt(2.0 / (9 * ci)), co * 9 * ci))
            parts.append(np.zeros(co))
        else:
            parts.append(np.zeros(co * 9 * ci))
            parts.append(np.array([0.0, 0.0, 0.0, gate_bias]))
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == gs.REPAIR_PARAMS
    return w


def scene_and_camera(kind: str, seed: int, n: int | None = None):
    """A seeded scene of the named distribution and its camera."""
    if kind == "object":
        scene = synth.scene_object_ground(seed, n or 500_000)
        cam = synth.centred_camera(1600, 1200, 1600.0)
        centre = np.array([0.0, 0.0, 2.0])
        radius = 2.0
    elif kind == "unbounded":
        scene = synth.scene_unbounded(seed, n or 1_500_000)
        cam = synth.centred_camera(1920, 1080, 1600.0)
        centre = np.zeros(3)
        radius = 3.0
    elif kind == "small":
        scene = synth.scene_slab_ball(seed)
        cam = synth.centred_camera(256, 192, 300.0)
        centre = np.array([0.0, 0.0, 3.0])
        radius = 3.0
    else:
        raise ValueError(kind)
    return scene, cam, centre, radius


def random_pose(rng, centre, radius, kind):
    """A head pose looking at the scene centre from a random direction on a band
    of yaw (+-30 deg) and pitch (+-10 deg)."""
    yaw = math.radians(rng.uniform(-30, 30))
    pitch = math.radians(rng.uniform(-10, 10))
    if kind == "small":  # stay in front of the slab
        eye = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2)])
        target = eye + np.array([math.sin(yaw) * 0.3, math.sin(pitch) * 0.3, 1.0])
        return synth.eye_pair(synth.look_at(eye, target))
    d = np.array([math.sin(yaw) * math.cos(pitch), math.sin(pitch), -math.cos(yaw) * math.cos(pitch)])
    return synth.eye_pair(synth.look_at(np.asarray(centre) + radius * d, centre))


class PairSet:
    """Resident training frames: features, target, interpolation-only image."""

    def __init__(self, ctx: gs.Context, cam, frames: int, device):
        H, W = cam.height, cam.width
        self.cam, self.ctx = cam, ctx
        self.feat = torch.zeros(frames, H, W, 8, dtype=torch.bfloat16, device=device)
        self.target = torch.zeros(frames, 3, H, W, device=device)
        self.plain = torch.zeros(frames, 3, H, W, device=device)
        self.tiles = []  # hole tiles: frame << 24 | ty << 12 | tx
        self.n = 0

    def add(self, ds, dom, aff):
        ctx, cam, k = self.ctx, self.cam, self.n
        interp = ctx.render_stereo(ds, dom, aff, cam, gap_thresh=2,
                                   roi=gs.roi_params(enable_center=0, repair_mode=3))
        self.plain[k].copy_(interp["rgb_aff"])
        ctx.repair_features(cam, out=self.feat[k])
        full = ctx.render_two_pass(ds, dom, aff, cam)
        self.target[k].copy_(full["rgb_aff"])
        # the tiles the network serves: holes outside the edge strips
        strip = (interp["cls_aff"] & gs.CLS_STRIP) > 0
        hole = (self.feat[k, :, :, 4].float() > 0.5) & ~strip
        H, W = cam.height, cam.width
        th = torch.nn.functional.max_pool2d(hole[None, None].float(), 16, 16, ceil_mode=True)[0, 0] > 0
        ys, xs = torch.nonzero(th, as_tuple=True)
        ids = (k << 24) | (ys.to(torch.int64) << 12) | xs.to(torch.int64)
        self.tiles.append(ids)
        self.n += 1

    def tile_tensor(self):
        return torch.cat(self.tiles).to(torch.int32)


def build_pairs(kind: str, scenes: int, poses_per_scene: int, seed: int, device, n_surfels=None):
    """Renders `scenes` x `poses_per_scene` pairs; returns (ctx, PairSet)."""
    rng = np.random.default_rng(seed)
    scene, cam, centre, radius = scene_and_camera(kind, seed, n_surfels)
    ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 26, device=device)
    pairs = PairSet(ctx, cam, scenes * poses_per_scene, device)
    for s in range(scenes):
        if s > 0:
            scene, _, _, _ = scene_and_camera(kind, seed + s, n_surfels)
        ds = gs.DeviceScene(scene, device=device)
        for _ in range(poses_per_scene):
            dom, aff = random_pose(rng, centre, radius, kind)
            pairs.add(ds, dom, aff)
    ctx.check_ok()
    return ctx, pairs


def save_checkpoint(path, ctx, next_step: int, generator: torch.Generator, meta: dict):
    """Everything a training run needs to continue exactly: FP32 parameters, both
    AdamW moments and their step count (from the context), the next step index,
    the state of the tile sampler's generator (the data cursor) and the run's
    settings (checked on resume)."""
    w, m, v, adam_steps = ctx.repair_state()
    tmp = f"{path}.tmp.npz"
    np.savez(tmp, weights=w, m=m, v=v, adam_steps=np.int64(adam_steps), next_step=np.int64(next_step),
             generator=generator.get_state().cpu().numpy(), meta=np.array(json.dumps(meta, sort_keys=True)))
    os.replace(tmp, path)


def load_checkpoint(path):
    z = np.load(path, allow_pickle=False)
    return {"weights": z["weights"], "m": z["m"], "v": z["v"], "adam_steps": int(z["adam_steps"]),
            "next_step": int(z["next_step"]), "generator": torch.from_numpy(z["generator"].copy()),
            "meta": json.loads(str(z["meta"]))}


def train(ctx: gs.Context, pairs: PairSet, steps: int, batch_tiles: int, lr: float, seed: int,
          weights: np.ndarray | None = None, log_every: int = 50, gate_weight: float = 1.0,
          checkpoint: str | None = None, checkpoint_every: int = 0, resume: str | None = None):
    """AdamW training on random batches of the pairs' hole tiles with a cosine
    rate decay. checkpoint / checkpoint_every: save the state every so many
    steps; resume: continue from a saved state (the same pairs and settings),
    which reproduces the uninterrupted run's remaining losses and final weights
    bit for bit ("{step}" in the checkpoint path is replaced by the step count).
    Returns (weights, [(step, loss, l1, bce, positive share)], seconds)."""
    all_tiles = pairs.tile_tensor()
    g = torch.Generator(device=all_tiles.device)
    g.manual_seed(seed)
    nb = min(batch_tiles, all_tiles.numel())
    meta = {"steps": steps, "batch_tiles": nb, "lr": lr, "seed": seed, "gate_weight": gate_weight,
            "hole_tiles": int(all_tiles.numel()), "frames": int(pairs.n)}
    start = 0
    if resume is not None:
        ck = load_checkpoint(resume)
        if ck["meta"] != meta:
            raise ValueError(f"checkpoint settings {ck['meta']} differ from this run's {meta}")
        ctx.repair_load_state(ck["weights"], ck["m"], ck["v"], ck["adam_steps"])
        g.set_state(ck["generator"])
        start = ck["next_step"]
    else:
        ctx.repair_load(weights if weights is not None else init_weights(seed))
    scratch = ctx.repair_scratch(nb)
    history = []
    t0 = time.time()
    for step in range(start, steps):
        pick = torch.randperm(all_tiles.numel(), generator=g, device=all_tiles.device)[:nb]
        tiles = all_tiles[pick].contiguous()
        # cosine decay to 10% of the rate
        lr_s = lr * (0.1 + 0.9 * 0.5 * (1 + math.cos(math.pi * step / max(steps - 1, 1))))
        loss = ctx.repair_train_step(pairs.feat, pairs.target, pairs.plain, tiles, scratch=scratch, lr=lr_s,
                                     gate_weight=gate_weight, want_loss=(step % log_every == 0 or step == steps - 1))
        if step % log_every == 0 or step == steps - 1:
            history.append((step, float(loss[0]), float(loss[1]), float(loss[2]), float(loss[3])))
        if checkpoint and checkpoint_every > 0 and (step + 1) % checkpoint_every == 0:
            save_checkpoint(checkpoint.format(step=step + 1), ctx, step + 1, g, meta)
    if all_tiles.is_cuda:
        torch.cuda.synchronize()
    return ctx.repair_read(0), history, time.time() - t0


def train_streamed(kind: str, n_scenes: int, poses_per_scene: int, shard_frames: int, epochs: int,
                   steps_per_shard: int, batch_tiles: int, lr: float, seed: int, device, n_surfels=None,
                   gate_weight: float = 1.0, log=print):
    """Training on more pairs than fit resident at once (the 2,000 pairs of 50
    scenes x 40 poses at 1920x1080 would take ~166 GB of frames): every epoch
    walks the pairs in shards of shard_frames frames, renders a shard (features,
    full render, interpolation-only image), and takes steps_per_shard AdamW steps
    on random batches of its hole tiles; the parameters and AdamW moments carry
    over between shards. The scenes stay resident; pair k is scene k //
    poses_per_scene at the k-th pose of a seeded sequence, the same in every
    epoch. Returns (weights, history, seconds)."""
    t0 = time.time()
    scenes = []
    for sidx in range(n_scenes):
        scene, cam, centre, radius = scene_and_camera(kind, seed + sidx, n_surfels)
        scenes.append(gs.DeviceScene(scene, device=device))
    n_pairs = n_scenes * poses_per_scene
    rng = np.random.default_rng(seed)
    poses = [random_pose(rng, centre, radius, kind) for _ in range(n_pairs)]
    ctx = gs.Context(max(sc.n for sc in scenes), cam.width, cam.height, max_instances=1 << 26, device=device)
    ctx.repair_load(init_weights(seed))
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    history, step = [], 0
    total_steps = epochs * ((n_pairs + shard_frames - 1) // shard_frames) * steps_per_shard
    scratch = ctx.repair_scratch(batch_tiles)
    for epoch in range(epochs):
        for s0 in range(0, n_pairs, shard_frames):
            pairs = PairSet(ctx, cam, min(shard_frames, n_pairs - s0), device)
            for k in range(s0, s0 + pairs.feat.shape[0]):
                pairs.add(scenes[k // poses_per_scene], *poses[k])
            all_tiles = pairs.tile_tensor()
            nb = min(batch_tiles, all_tiles.numel())
            for _ in range(steps_per_shard):
                pick = torch.randperm(all_tiles.numel(), generator=g, device=device)[:nb]
                lr_s = lr * (0.1 + 0.9 * 0.5 * (1 + math.cos(math.pi * step / max(total_steps - 1, 1))))
                want = step % 100 == 0 or step == total_steps - 1
                loss = ctx.repair_train_step(pairs.feat, pairs.target, pairs.plain, all_tiles[pick].contiguous(),
                                             scratch=scratch if nb == batch_tiles else None, lr=lr_s,
                                             gate_weight=gate_weight, want_loss=want)
                if want:
                    history.append((step, float(loss[0]), float(loss[1]), float(loss[2]), float(loss[3])))
                    log(f"epoch {epoch} pairs {s0}-{s0 + pairs.n - 1} step {step} loss {loss[0]:.5f} "
                        f"hole tiles {all_tiles.numel()}")
                step += 1
            del pairs, all_tiles
    ctx.check_ok()
    torch.cuda.synchronize()
    return ctx.repair_read(0), history, time.time() - t0


def psnr(a, b) -> float:
    mse = torch.mean((a - b) ** 2).item()
    return 10 * math.log10(1.0 / max(mse, 1e-20))


def evaluate(ctx: gs.Context, kind: str, seeds, poses_per_scene: int, seed: int, tau: float, device,
             n_surfels=None):
    """Held-out frames: PSNR against the full render of the plain method, of the
    learned repair, and of the interpolation-only fill; hole-pixel L1 of the
    network fill and of the interpolation fill; share of ROI tiles the gate took
    out of the re-render."""
    rng = np.random.default_rng(seed)
    rows = []
    for sd in seeds:
        scene, cam, centre, radius = scene_and_camera(kind, sd, n_surfels)
        ds = gs.DeviceScene(scene, device=device)
        H, W = cam.height, cam.width
        fill = torch.zeros(1, 3, H, W, device=device)
        for _ in range(poses_per_scene):
            dom, aff = random_pose(rng, centre, radius, kind)
            full = {k: v.clone() for k, v in ctx.render_two_pass(ds, dom, aff, cam).items()}
            interp = {k: v.clone() for k, v in
                      ctx.render_stereo(ds, dom, aff, cam, gap_thresh=2, roi=gs.roi_params(enable_center=0)).items()}
            plain = {k: v.clone() for k, v in ctx.render_stereo(ds, dom, aff, cam, gap_thresh=2).items()}
            ctx.render_stereo(ds, dom, aff, cam, gap_thresh=2, roi=gs.roi_params(repair_mode=3))
            feat = ctx.repair_features(cam)
            learned = {k: v.clone() for k, v in ctx.render_stereo(
                ds, dom, aff, cam, gap_thresh=2, roi=gs.roi_params(repair_mode=1, gate_tau=tau)).items()}
            ty, tx = (H + 15) // 16, (W + 15) // 16
            tiles = torch.tensor([(y << 12) | x for y in range(ty) for x in range(tx)], dtype=torch.int32,
                                 device=device)
            ctx.repair_infer(feat[None], tiles, fill=fill)
            strip = (plain["cls_aff"] & gs.CLS_STRIP) > 0
            hole = (feat[:, :, 4].float() > 0.5) & ~strip  # holes the method fills itself
            tgt = full["rgb_aff"]
            base = feat[:, :, :3].float().permute(2, 0, 1)
            l1_net = (torch.clamp(fill[0], min=0) - tgt).abs()[:, hole].mean().item() if hole.any() else 0.0
            # the method's fill of the same holes (the network's starting point)
            l1_interp = (base - tgt).abs()[:, hole].mean().item() if hole.any() else 0.0
            roi_plain = ((plain["cls_aff"] & gs.CLS_RENDER) > 0).float().mean().item()
            roi_learned = ((learned["cls_aff"] & gs.CLS_RENDER) > 0).float().mean().item()
            net_px = ((learned["cls_aff"] & gs.CLS_NET) > 0).float().mean().item()
            rows.append(dict(psnr_plain=psnr(plain["rgb_aff"], tgt), psnr_learned=psnr(learned["rgb_aff"], tgt),
                             psnr_interp=psnr(interp["rgb_aff"], tgt), l1_net=l1_net, l1_interp=l1_interp,
                             roi_plain=roi_plain, roi_learned=roi_learned, net_pixels=net_px))
    ctx.check_ok()
    return {k: float(np.mean([r[k] for r in rows])) for k in rows[0]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scene", default="object", choices=["object", "unbounded", "small"])
    ap.add_argument("--scenes", type=int, default=4)
    ap.add_argument("--poses", type=int, default=6)
    ap.add_argument("--surfels", type=int, default=None)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--gate-weight", type=float, default=1.0)
    ap.add_argument("--seed", type=int, default=7000)
    ap.add_argument("--out", required=True)
    ap.add_argument("--checkpoint", default=None, help="save the training state here every --checkpoint-every steps")
    ap.add_argument("--checkpoint-every", type=int, default=0)
    ap.add_argument("--resume", default=None, help="continue from a saved training state")
    ap.add_argument("--shard", type=int, default=0,
                    help="stream the pairs in shards of this many frames (rendered on the fly), for pair counts "
                         "that do not fit resident; --steps is then per shard and --epochs passes are made")
    ap.add_argument("--epochs", type=int, default=1)
    ap.add_argument("--eval-scenes", type=int, default=0,
                    help="after training, evaluate on this many held-out scene seeds (3 poses each)")
    ap.add_argument("--tau", type=float, default=0.5)
    args = ap.parse_args()
    dev = torch.device("cuda", 0)
    from . import build
    build.build()
    if args.shard > 0:
        w, hist, secs = train_streamed(args.scene, args.scenes, args.poses, args.shard, args.epochs, args.steps,
                                       args.batch, args.lr, args.seed, dev, args.surfels,
                                       gate_weight=args.gate_weight)
        np.save(args.out, w)
        print(f"trained on {args.scenes * args.poses} pairs in shards of {args.shard}, {args.epochs} epochs, "
              f"{len(hist)} logged steps, {secs:.1f} s")
        if args.eval_scenes:
            _report_eval(args, w, dev)
        return
    ctx, pairs = build_pairs(args.scene, args.scenes, args.poses, args.seed, dev, args.surfels)
    w, hist, secs = train(ctx, pairs, args.steps, args.batch, args.lr, args.seed, gate_weight=args.gate_weight,
                          checkpoint=args.checkpoint, checkpoint_every=args.checkpoint_every, resume=args.resume)
    np.save(args.out, w)
    for h in hist:
        print(f"step {h[0]:5d} loss {h[1]:.5f} l1 {h[2]:.5f} bce {h[3]:.5f} pos {h[4]:.3f}")
    print(f"trained {args.steps} steps in {secs:.1f} s on {pairs.n} frames, {pairs.tile_tensor().numel()} hole tiles")
    if args.eval_scenes:
        _report_eval(args, w, dev)


def _report_eval(args, w, dev):
    """Held-out scene seeds lie above every training seed."""
    scene, cam, _, _ = scene_and_camera(args.scene, args.seed, args.surfels)
    ctx = gs.Context(scene.n, cam.width, cam.height, max_instances=1 << 26, device=dev)
    ctx.repair_load(w)
    seeds = [args.seed + 100000 + i for i in range(args.eval_scenes)]
    ev = evaluate(ctx, args.scene, seeds, 3, args.seed + 1, args.tau, dev, args.surfels)
    print("eval " + " ".join(f"{k}={v:.4f}" for k, v in ev.items()))


if __name__ == "__main__":
    main()
