"""Shared helpers for the parity tests: build seeded inputs, move them to the GPU, run the oracle,
compare with the tolerances of the method (relative 1e-4 in FP32, 2e-3 for the compact / FP16
path, 8-bit within 1 LSB)."""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass

import numpy as np

import oracle
import synth

REL_TOL_FP32 = 1e-4
REL_TOL_REDUCED = 2e-3


@dataclass
class Inputs:
    cfg: dict
    scene: synth.Scene
    g: synth.GBuffer
    env: np.ndarray
    kernel: np.ndarray
    noise: np.ndarray
    W: int
    H: int

    @property
    def lights(self):
        return self.scene.lights

    def compact(self):
        return synth.encode_compact(self.g)


def make_inputs(name: str, W: int | None = None, H: int | None = None, spheres: int | None = None,
                lights: int | None = None, env_seed: int | None = None) -> Inputs:
    cfg = dict(synth.CONFIGS[name])
    W = W or cfg["width"]
    H = H or cfg["height"]
    sc = synth.make_scene(cfg["seed"], W, H, spheres if spheres is not None else cfg["spheres"],
                          lights if lights is not None else cfg["lights"])
    g = synth.raycast_gbuffer(sc)
    We, He = cfg["env"]
    env = synth.make_env(cfg["seed"] if env_seed is None else env_seed, We, He)
    k = synth.make_ssao_kernel(cfg["seed"], cfg["ssao_k"])
    nz = synth.make_ssao_noise(cfg["seed"])
    return Inputs(cfg, sc, g, env, k, nz, W, H)


@functools.lru_cache(maxsize=4)
def _oracle_ibl_cached(key, env_bytes, shape, M, N, S, NL, Wi, Hi):
    env = np.frombuffer(env_bytes, np.float32).reshape(shape)
    return oracle.precompute_ibl(env, M, N, S, NL, Wi, Hi)


def oracle_ibl(inp: Inputs) -> oracle.IblSet:
    c = inp.cfg
    Wi, Hi = c["irr"]
    return _oracle_ibl_cached((c["seed"], inp.env.shape), inp.env.tobytes(), inp.env.shape, c["levels"],
                              c["prefilter_samples"], c["lut"], c["lut_samples"], Wi, Hi)


def oracle_camera(inp: Inputs):
    return oracle.camera(inp.scene.camera_array(), inp.scene.fov_y, inp.W, inp.H)


def rel_err(gpu: np.ndarray, ref: np.ndarray, tau: float) -> np.ndarray:
    """Per channel |g - o| / max(|o|, tau)."""
    return np.abs(gpu - ref) / np.maximum(np.abs(ref), tau)


def luminance_tau(ref: np.ndarray) -> float:
    lum = 0.2126 * ref[..., 0] + 0.7152 * ref[..., 1] + 0.0722 * ref[..., 2]
    return 1e-3 * float(np.mean(lum))


def ulp_perturbations(gb_px: np.ndarray, steps=(-2, 2)):
    """Copies of decoded G-buffer rows (n, 9) with depth and each normal component moved by
    `steps` float32 ulps, one quantity at a time."""
    out = []
    for col in (4, 5, 6, 8):
        for s in steps:
            p = gb_px.copy()
            v = p[:, col].astype(np.float32)
            for _ in range(abs(s)):
                v = np.nextafter(v, np.float32(np.inf) if s > 0 else np.float32(-np.inf))
            p[:, col] = v.astype(np.float64)
            out.append((col, p))
    return out


def shade_conditioning(gb: np.ndarray, cam, lights, ibl, flags, ao, ao_scale, pixels, tau, base):
    """Largest relative change of the oracle's output at `pixels` when an input moves by 2 ulps:
    how much of a GPU/oracle difference rounding alone can explain."""
    H, W = gb.shape[:2]
    flat = gb.reshape(-1, 9)
    spread = np.zeros(len(pixels))
    for col, rows in ulp_perturbations(flat[pixels]):
        gb2 = flat.copy()
        gb2[pixels] = rows
        o2 = oracle.shade(gb2.reshape(H, W, 9), cam, lights, ibl, flags, ao=ao, ao_scale=ao_scale,
                          pixels=pixels)
        spread = np.maximum(spread, rel_err(o2, base, tau).max(axis=1))
    return spread


def check_hdr(gpu: np.ndarray, ref: np.ndarray, tol: float, gb=None, cam=None, lights=None, ibl=None,
              flags=None, ao=None, ao_scale=1, pixels=None, max_ill_share=1e-3, report=None):
    """Parity rule for linear HDR: every channel within `tol` relative (floor tau), except
    ill-conditioned pixels (oracle moves by more than tol/2 under 2-ulp input perturbations),
    whose share must stay below `max_ill_share`."""
    tau = luminance_tau(ref)
    e = rel_err(gpu, ref, tau).max(axis=-1).reshape(-1)
    bad = np.nonzero(e > tol)[0]
    ill = 0
    if len(bad) and gb is not None:
        px = bad if pixels is None else np.asarray(pixels)[bad]
        spread = shade_conditioning(gb, cam, lights, ibl, flags, ao, ao_scale, px, tau,
                                    ref.reshape(-1, 3)[bad])
        still = bad[spread <= 0.5 * tol]
        ill = len(bad) - len(still)
        bad = still
    if report is not None:
        report.update(max_rel=float(e.max()), ill=ill, n=int(e.size),
                      max_rel_well=float(np.delete(e, np.nonzero(e > tol)[0]).max() if e.size else 0))
    assert len(bad) == 0, f"{len(bad)} pixels beyond {tol}: worst {e[bad].max():.3g} at {bad[:5]}"
    assert ill <= max_ill_share * e.size, f"{ill} ill-conditioned pixels of {e.size}"


def check_ldr(gpu: np.ndarray, ref: np.ndarray, scaled: np.ndarray, min_exact=0.999):
    """8-bit rule: every channel within 1 LSB, at least `min_exact` of pixels identical, and
    exact wherever the oracle's unrounded value is not within 1e-3 of a rounding boundary."""
    g = gpu[..., :3].reshape(-1, 3).astype(np.int32)
    o = ref[..., :3].reshape(-1, 3).astype(np.int32)
    d = np.abs(g - o)
    assert d.max() <= 1, f"max LSB difference {d.max()}"
    exact = (d == 0).all(axis=1).mean()
    assert exact >= min_exact, f"only {exact:.5f} of pixels identical"
    frac = scaled.reshape(-1, 3) + 0.5
    near = np.abs(frac - np.round(frac)) < 1e-3
    assert (d[~near] == 0).all(), "difference away from a rounding boundary"
    assert (gpu[..., 3] == 255).all()
    return exact


def sample_pixels(W: int, H: int, n: int, seed: int = 0, depth=None):
    """Seeded pixel subset that always contains the four corners and the last row."""
    rng = np.random.default_rng(seed)
    px = set(rng.choice(W * H, size=min(n, W * H), replace=False).tolist())
    px |= {0, W - 1, (H - 1) * W, H * W - 1}
    px |= set(((H - 1) * W + np.arange(0, W, max(1, W // 64))).tolist())
    return np.array(sorted(px), np.int64)


def ao_tie_check(gpu: np.ndarray, ao: np.ndarray, lo: np.ndarray, hi: np.ndarray, tol: float = 1e-4):
    """AO parity with ties: where no decision is near its threshold (lo == hi) the values agree
    within tol; elsewhere the GPU value lies within [lo - tol, hi + tol]."""
    g = gpu.reshape(-1)
    a, l, h = ao.reshape(-1), lo.reshape(-1), hi.reshape(-1)
    unique = l == h
    assert np.all(np.abs(g[unique] - a[unique]) <= tol), \
        f"max AO diff {np.abs(g[unique] - a[unique]).max():.3g}"
    assert np.all((g >= l - tol) & (g <= h + tol))
    return float(unique.mean())


def gpu_inputs(inp: Inputs, compact: bool = False, device="cuda"):
    """Tensors and structs for the CUDA path (the binding)."""
    import torch

    import paper_2012_03325_gb300 as ep
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    if compact:
        c = inp.compact()
        gb = ep.GBuffer.compact(t(c.rt0), t(c.rt1), t(c.rt2), t(c.depth))
    else:
        gb = ep.GBuffer.fp32(t(inp.g.rt0), t(inp.g.rt1), t(inp.g.depth))
    cam = ep.camera(inp.scene.camera_array(), inp.scene.fov_y, inp.W, inp.H)
    return dict(gb=gb, cam=cam, lights=t(inp.lights), env=t(inp.env), kernel=t(inp.kernel),
                noise=t(inp.noise))


def gpu_ibl(inp: Inputs, env_t, stream=None):
    import paper_2012_03325_gb300 as ep
    c = inp.cfg
    p = ep.ibl_params(c["levels"], c["prefilter_samples"], c["lut"], c["lut_samples"], *c["irr"])
    ibl = ep.Ibl(p, inp.env.shape[1], inp.env.shape[0])
    ep.epbr_precompute_ibl(env_t, ibl, stream=stream)
    return ibl


def decoded(inp: Inputs, compact: bool = False) -> np.ndarray:
    if compact:
        c = inp.compact()
        return oracle.decode_compact(c.rt0, c.rt1, c.rt2, c.depth)
    return oracle.decode_fp32(inp.g.rt0, inp.g.rt1, inp.g.depth)


def fp16_round(x: np.ndarray) -> np.ndarray:
    return np.clip(x, -65504, 65504).astype(np.float16).astype(np.float64)


__all__ = [n for n in dir() if not n.startswith("_")] + ["math"]
