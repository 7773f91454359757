"""Error report of the CUDA path against the FP64 oracle, per workload (needs a GPU).

For each configuration: HDR relative error per channel (metric: |g - o| / max(|o|, tau),
tau = 1e-3 x mean oracle luminance) as max / p99.9 / mean over the checked pixels, the share of
ill-conditioned pixels, AO error where no decision is tied, and the 8-bit LSB histogram.
  small        256x256, FP32 G-buffer, RGBA32F, every pixel
  full         1920x1080, FP32 G-buffer, RGBA32F, 20000 sampled pixels
  uhd_compact  3840x2160, compact G-buffer (14 B/px), RGBA16F, 20000 sampled pixels
Writes one JSON object per line to stdout.

  python tests/report_errors.py [--pixels 20000]
"""
import argparse
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
import synth  # noqa: E402
from _common import (REL_TOL_FP32, REL_TOL_REDUCED, decoded, gpu_ibl, gpu_inputs, luminance_tau,  # noqa: E402
                     make_inputs, oracle_camera, rel_err, sample_pixels, shade_conditioning)


def report(name, n_px):
    import torch

    import paper_2012_03325_gb300 as ep
    compact = name == "uhd_compact"
    inp = make_inputs(name, env_seed=synth.CONFIGS["full"]["seed"] if compact else None)
    d = gpu_inputs(inp, compact=compact)
    ibl = gpu_ibl(inp, d["env"])
    c = inp.cfg
    ref_ibl = oracle.precompute_ibl(inp.env, c["levels"], c["prefilter_samples"], c["lut"], c["lut_samples"],
                                    *c["irr"])
    sp = ep.SsaoParams(d["kernel"], d["noise"], radius=c["radius"], scale=2, blur_radius=c["blur"])
    Ha, Wa = sp.ao_shape(inp.W, inp.H)
    ao = torch.zeros(Ha, Wa, device="cuda")
    ep.epbr_ssao(d["gb"], d["cam"], sp, ao)
    ao_in = synth.make_ao_field(5, Wa, Ha)
    fmt = ep.EPBR_HDR_RGBA16F if compact else ep.EPBR_HDR_RGBA32F
    hdr = torch.zeros(inp.H, inp.W, 4, dtype=torch.float16 if compact else torch.float32, device="cuda")
    ldr = torch.zeros(inp.H, inp.W, 4, dtype=torch.uint8, device="cuda")
    ep.epbr_shade_tonemap(d["gb"], d["cam"], d["lights"], ibl,
                          ep.shade_params(ep.EPBR_SHADE_ALL, torch.from_numpy(ao_in).cuda(), 2), hdr, fmt,
                          ep.tonemap_params(), ldr)
    torch.cuda.synchronize()
    gb = decoded(inp, compact)
    cam = oracle_camera(inp)
    px = None if name == "small" else sample_pixels(inp.W, inp.H, n_px, seed=11)
    o = oracle.shade(gb, cam, inp.lights, ref_ibl, ep.EPBR_SHADE_ALL, ao=ao_in, ao_scale=2, pixels=px)
    o = o.reshape(-1, 3)
    g = hdr.cpu().numpy().astype(np.float64)[..., :3].reshape(-1, 3)
    if px is not None:
        g = g[px]
    tau = luminance_tau(o)
    e = rel_err(g, o, tau).max(axis=1)
    tol = REL_TOL_REDUCED if compact else REL_TOL_FP32
    bad = np.nonzero(e > tol)[0]
    ill = 0
    if len(bad):
        pix = bad if px is None else px[bad]
        spread = shade_conditioning(gb, cam, inp.lights, ref_ibl, ep.EPBR_SHADE_ALL, ao_in, 2, pix, tau, o[bad])
        ill = int(np.sum(spread > 0.5 * tol))
    out8, _ = oracle.tonemap(o)
    g8 = ldr.cpu().numpy().reshape(-1, 4)
    if px is not None:
        g8 = g8[px]
    lsb = np.abs(g8[:, :3].astype(int) - out8[:, :3].astype(int)).max(axis=1)
    ao_px = sample_pixels(Wa, Ha, min(n_px, Wa * Ha), seed=12) if name != "small" else None
    a, lo, hi = oracle.ssao(gb, cam, K=c["ssao_k"], scale=2, radius=c["radius"], bias=0.05 * c["radius"],
                            blur_radius=c["blur"], sigma_s=2.0, sigma_z=0.1, kernel=inp.kernel, noise=inp.noise,
                            blurred=True, texels=ao_px)
    ga = ao.cpu().numpy().reshape(-1)
    if ao_px is not None:
        ga = ga[ao_px]
    a, lo, hi = a.reshape(-1), lo.reshape(-1), hi.reshape(-1)
    uniq = lo == hi
    return {"workload": name, "size": f"{inp.W}x{inp.H}", "gbuffer": "compact 14 B/px" if compact else "fp32 36 B/px",
            "hdr": "RGBA16F" if compact else "RGBA32F", "pixels_checked": int(e.size),
            "hdr_rel_err": {"max": float(e.max()), "p99.9": float(np.percentile(e, 99.9)), "mean": float(e.mean())},
            "tolerance": tol, "beyond_tolerance": int(len(bad)), "ill_conditioned": ill,
            "ldr_lsb_hist": {str(k): int(np.sum(lsb == k)) for k in range(int(lsb.max()) + 1)},
            "ao_abs_err_untied": {"max": float(np.abs(ga[uniq] - a[uniq]).max()), "untied_share": float(uniq.mean())},
            "ao_in_tie_interval": bool(np.all((ga >= lo - 1e-4) & (ga <= hi + 1e-4)))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pixels", type=int, default=20000)
    ap.add_argument("--workloads", default="small,full,uhd_compact")
    args = ap.parse_args()
    for name in args.workloads.split(","):
        print(json.dumps(report(name, args.pixels)), flush=True)


if __name__ == "__main__":
    main()
