"""Per-configuration measurements behind the results table of the baseline
notes: GPU throughput of each configuration (CUDA events around the library
call, inputs resident in device memory, best of several runs) and quality
against the FP64 oracle on the same seeded synthetic images.  Not a test
(pytest does not collect it); run on a GPU machine:

    python tests/measure_configs.py [--quick]

Prints one JSON object.  Configurations (image seeds as in the input recipe):
  cfg1  BM3D FP32, one 128 x 128 grey image, sigma 25
  cfg2  NL-means and BM3D on 8 grey 512 x 512 images, sigma 15 / 25 / 50
  cfg3  BM3D on 16 grey 1024 x 1024 images, sigma 25: FP32, BF16 transforms,
        BF16 transforms + BF16 matching prefilter (oracle on a 256 x 256 crop)
  cfg4  hybrid BM3D + 10x32 CNN on the 32 held-out 512 x 512 images, sigma 25
"""
import argparse
import json
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def gpu_ms(fn, reps=5):
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="oracle on one image per configuration only")
    ap.add_argument("--only", default="cfg1,cfg2,cfg3,cfg4", help="comma-separated configurations to run")
    args = ap.parse_args()
    want = set(args.only.split(","))
    import oracle
    from paper_2403_03488_gb300 import api as A, synth
    oracle.build()
    torch.cuda.set_device(0)
    res = {"oracle_threads": oracle.num_threads()}
    P32 = A.default_bm3d_params(precision=A.DN_FP32)
    P16 = A.default_bm3d_params(precision=A.DN_BF16)
    P16M = A.default_bm3d_params(precision=A.DN_BF16 | A.DN_BF16_MATCH)

    if "cfg1" in want:
        cfg1(A, oracle, synth, P32, res)
    if "cfg2" in want:
        cfg2(A, oracle, synth, P32, P16, res, args.quick)
    if "cfg3" in want:
        cfg3(A, oracle, synth, P32, P16, P16M, res)
    if "cfg4" in want:
        cfg4(A, oracle, synth, P32, P16, res)
    res["device_error"] = A.device_error()
    print(json.dumps(res, indent=1, default=float))


def cfg1(A, oracle, synth, P32, res):
    clean, noisy = synth.make_batch([0], 128, 128, 25.0)
    x = torch.from_numpy(noisy).cuda()
    ms = gpu_ms(lambda: A.denoise_bm3d(x, 25.0, P32), reps=20)
    out = A.denoise_bm3d(x, 25.0, P32).cpu().numpy()[0]
    t0 = time.perf_counter()
    _, ref = oracle.bm3d(noisy[0], 25.0)
    to = time.perf_counter() - t0
    res["cfg1"] = {"fp32_mpix_s": 128 * 128 / 1e3 / ms, "dpsnr_vs_fp64_db": oracle.psnr(out, clean[0]) -
                   oracle.psnr(ref, clean[0]), "max_abs_err": float(np.abs(out - ref).max()),
                   "oracle_mpix_s": 128 * 128 / 1e6 / to}



def cfg2(A, oracle, synth, P32, P16, res, quick):
    c2 = {}
    for s in (15.0, 25.0, 50.0):
        clean, noisy = synth.make_batch(range(8), 512, 512, s)
        x = torch.from_numpy(noisy).cuda()
        mp = 8 * 512 * 512 / 1e6
        row = {"nlm_mpix_s": mp / gpu_ms(lambda: A.denoise_nlm(x, s)) * 1e3,
               "bm3d_fp32_mpix_s": mp / gpu_ms(lambda: A.denoise_bm3d(x, s, P32)) * 1e3,
               "bm3d_bf16_mpix_s": mp / gpu_ms(lambda: A.denoise_bm3d(x, s, P16)) * 1e3}
        on = A.denoise_nlm(x, s).cpu().numpy()
        o32 = A.denoise_bm3d(x, s, P32).cpu().numpy()
        o16 = A.denoise_bm3d(x, s, P16).cpu().numpy()
        imgs = range(1) if quick else range(8)
        dn, db, d16, en, eb, e16, tn, tb = [], [], [], [], [], [], 0.0, 0.0
        for i in imgs:
            t0 = time.perf_counter()
            rn = oracle.nlm_image(noisy[i], s)
            tn += time.perf_counter() - t0
            t0 = time.perf_counter()
            _, rb = oracle.bm3d(noisy[i], s)
            tb += time.perf_counter() - t0
            pc = lambda o: oracle.psnr(o, clean[i])
            dn.append(pc(on[i]) - pc(rn))
            db.append(pc(o32[i]) - pc(rb))
            d16.append(pc(o16[i]) - pc(rb))
            en.append(float(np.abs(on[i] - rn).max()))
            eb.append(float(np.abs(o32[i] - rb).max()))
            e16.append(float(np.abs(o16[i] - rb).max()))
        k = len(dn)
        row.update({"nlm_dpsnr_db_max": float(np.max(np.abs(dn))), "nlm_max_abs_err": max(en),
                    "bm3d_fp32_dpsnr_db_mean": float(np.mean(db)), "bm3d_fp32_max_abs_err": max(eb),
                    "bm3d_bf16_dpsnr_db_mean": float(np.mean(d16)), "bm3d_bf16_max_abs_err": max(e16),
                    "oracle_images": k, "oracle_nlm_mpix_s": k * 0.262144 / tn,
                    "oracle_bm3d_mpix_s": k * 0.262144 / tb})
        c2["sigma%d" % int(s)] = row
    res["cfg2"] = c2


def cfg3(A, oracle, synth, P32, P16, P16M, res):
    clean, noisy = synth.make_batch(range(100, 116), 1024, 1024, 25.0)
    x = torch.from_numpy(noisy).cuda()
    mp = 16 * 1024 * 1024 / 1e6
    c3 = {}
    outs = {}
    for name, p in (("fp32", P32), ("bf16", P16), ("bf16_match", P16M)):
        c3[name + "_mpix_s"] = mp / gpu_ms(lambda: A.denoise_bm3d(x, 25.0, p), reps=3) * 1e3
        outs[name] = A.denoise_bm3d(x, 25.0, p).cpu().numpy()
    c3["bf16_match_equals_bf16"] = bool(np.array_equal(outs["bf16"], outs["bf16_match"]))
    c3["bf16_minus_fp32_psnr_db_mean"] = float(np.mean([oracle.psnr(outs["bf16"][i], clean[i]) -
                                                        oracle.psnr(outs["fp32"][i], clean[i]) for i in range(16)]))
    crop_c, crop_n = clean[0, :, :256, :256], noisy[0, :, :256, :256]
    xc = torch.from_numpy(np.ascontiguousarray(crop_n[None])).cuda()
    t0 = time.perf_counter()
    _, rc = oracle.bm3d(crop_n, 25.0)
    c3["oracle_mpix_s_crop"] = 0.065536 / (time.perf_counter() - t0)
    for name, p in (("fp32", P32), ("bf16", P16)):
        oc = A.denoise_bm3d(xc, 25.0, p).cpu().numpy()[0]
        c3[name + "_crop_dpsnr_vs_fp64_db"] = oracle.psnr(oc, crop_c) - oracle.psnr(rc, crop_c)
        c3[name + "_crop_max_abs_err"] = float(np.abs(oc - rc).max())
    res["cfg3"] = c3


def cfg4(A, oracle, synth, P32, P16, res):
    from bench import load_weights
    w, wsrc = load_weights(torch.device("cuda", 0))
    clean, noisy = synth.make_batch(range(5000, 5032), 512, 512, 25.0)
    x = torch.from_numpy(noisy).cuda()
    mp = 32 * 512 * 512 / 1e6
    c4 = {"weights": wsrc}
    for name, bp, cp in (("fp32_plain", P32, A.DN_FP32), ("default", P32, A.DN_BF16), ("bf16", P16, A.DN_BF16)):
        run = lambda: A.denoise_hybrid(x, 25.0, w, prefilter_params=bp, cnn_precision=cp)
        c4[name + "_mpix_s"] = mp / gpu_ms(run, reps=3) * 1e3
        o = run().cpu().numpy()
        c4[name + "_psnr_db"] = float(np.mean([oracle.psnr(o[i], clean[i]) for i in range(32)]))
    ob = A.denoise_bm3d(x, 25.0, P32).cpu().numpy()
    c4["bm3d_only_psnr_db"] = float(np.mean([oracle.psnr(ob[i], clean[i]) for i in range(32)]))
    res["cfg4"] = c4


if __name__ == "__main__":
    main()
