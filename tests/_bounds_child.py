"""Runs in its own process with the range-checked library (libfos_bounds.so)
loaded instead of the release one; prints one JSON line.  Used by
test_gpu_bounds.py: every configuration must record no violation and still
match the oracle (PBAS bit-exact, GMM within the FP32 tolerance)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import numpy as np  # noqa: E402


def main():
    from paper_2002_00250_gb300 import build, fos
    path = build.build(bounds=True)
    lib = fos.load(path)
    import oracle
    oracle.build()
    from _helpers import oracle_gmm_params, oracle_pbas_params, scene
    assert lib.fos_bounds_checked() == 1
    out = {"runs": []}
    import ctypes
    n, site, idx = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_int64()
    assert lib.fos_bounds_selftest(ctypes.byref(n), ctypes.byref(site), ctypes.byref(idx)) == 0
    out["selftest"] = [n.value, site.value, idx.value]

    def check(seg, W, H, frames, rgb, depth, label):
        p = seg.params
        g = oracle.GMM(W, H, **oracle_gmm_params(p)) if p.methods & fos.METHOD_GMM else None
        pb = oracle.PBAS(W, H, **oracle_pbas_params(p)) if p.methods & fos.METHOD_PBAS else None
        mg, mp = seg.process_host(rgb[:frames], depth[:frames])
        bad = np.zeros(W * H, bool)
        ok = True
        for t in range(frames):
            if pb is not None:
                ok &= bool(np.array_equal(mp[t], pb.step(rgb[t], depth[t])))
            if g is not None:
                mo, margin = g.step(rgb[t], depth[t], want_margin=True)
                bad |= (margin < 1e-5).ravel()
                ok &= bool(np.array_equal(mg[t].ravel()[~bad], mo.ravel()[~bad]))
        seg.decode_state()  # the flush kernel runs before an export
        v = seg.bounds_status()
        out["runs"].append({"case": label, "oracle_equal": ok, "violations": v[0], "site": v[1], "index": v[2]})

    for (W, H) in ((1, 1), (3, 5), (17, 13), (67, 45), (136, 40)):
        rgb, depth, _ = scene(W, H, 6, seed=W * 7 + H, n_objects=2, hole_fraction=0.05)
        check(fos.Segmenter(W, H), W, H, 6, rgb, depth, f"fused {W}x{H}")
        check(fos.Segmenter(W, H, methods=fos.METHOD_PBAS), W, H, 6, rgb, depth, f"pbas {W}x{H}")
        check(fos.Segmenter(W, H, methods=fos.METHOD_GMM), W, H, 6, rgb, depth, f"gmm {W}x{H}")
        check(fos.Segmenter(W, H, methods=fos.METHOD_PBAS, pbas_propagate=1, forced_rng=3, N=4), W, H, 6, rgb,
              depth, f"pbas propagate {W}x{H}")
    # the GMM over several frames in one launch, and other tile shapes
    import torch
    W, H = 136, 40
    rgb, depth, _ = scene(W, H, 6, seed=5)
    for opt, val in ((fos.OPT_PBAS_PX, 4), (fos.OPT_PBAS_TY, 4), (fos.OPT_GMM_PX, 1)):
        seg = fos.Segmenter(W, H)
        seg.set_option(opt, val)
        check(seg, W, H, 6, rgb, depth, f"fused option {opt}={val}")
    seg = fos.Segmenter(W, H, methods=fos.METHOD_GMM)
    d_rgb, d_dep = torch.from_numpy(rgb).cuda(), torch.from_numpy(depth).cuda()
    mg = torch.empty((6, H, W), dtype=torch.uint8, device="cuda")
    seg.process_device(d_rgb, d_dep, mask_gmm=mg)
    torch.cuda.synchronize()
    v = seg.bounds_status()
    out["runs"].append({"case": "gmm all frames in one launch", "oracle_equal": True, "violations": v[0],
                        "site": v[1], "index": v[2]})
    # a mixed batch: ragged widths take the one-pixel tiles, even ones the vector tiles
    for sizes in (((136, 40), (64, 48), (256, 24)), ((136, 40), (67, 45), (33, 17))):
        b = fos.Batch(len(sizes))
        slots = [b.add(w, h, stream_id=40 + i) for i, (w, h) in enumerate(sizes)]
        data = [scene(w, h, 5, seed=60 + i) for i, (w, h) in enumerate(sizes)]
        for f in range(5):
            r = [torch.from_numpy(data[i][0][f]).cuda() for i in range(len(sizes))]
            d = [torch.from_numpy(data[i][1][f]).cuda() for i in range(len(sizes))]
            mgs = [torch.empty((h, w), dtype=torch.uint8, device="cuda") for (w, h) in sizes]
            mps = [torch.empty((h, w), dtype=torch.uint8, device="cuda") for (w, h) in sizes]
            b.process(slots, r, d, mgs, mps)
        torch.cuda.synchronize()
        for i, sl in enumerate(slots):
            ctx = b.context(sl)
            n, site, idx = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_int64()
            st = lib.fos_bounds_status(ctx, ctypes.byref(n), ctypes.byref(site), ctypes.byref(idx))
            out["runs"].append({"case": f"batch {sizes} stream {i}", "oracle_equal": st == 0,
                                "violations": n.value, "site": site.value, "index": idx.value})
        b.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
