"""Tolerances of the replay comparisons, derived from the arithmetic they compare."""
import numpy as np

U = 2.0 ** -24  # unit roundoff of float32
# An FP32 hit distance agrees with the FP64 one to max(1e-5 t, T_ERR_K * terr), terr being the
# oracle's error scale of the winning hit (4 rounding units of the coordinate magnitude over
# the ray's obliquity); an FP32 t passes through about 16 such roundings.
T_ERR_K = 4.0


def spawn_tolerance(o, d, t, o_next):
    """Per-component bound on the difference between two spawn points of the same hit,
    o + t d offset along the normal, one computed in FP64 from float inputs and one in FP32
    (or captured as float): at most two roundings of o + t d (product and sum) and one of
    the offset sum, each within u = 2^-24 of its magnitude, doubled for margin."""
    o = np.asarray(o, np.float64)
    d = np.asarray(d, np.float64)
    t = np.asarray(t, np.float64)[..., None]
    return 4.0 * U * (np.abs(o) + np.abs(t * d) + np.abs(np.asarray(o_next, np.float64)))


def scenes_mat_ggx():
    from paper_2310_07182_gb300 import scenes
    return scenes.MAT_GGX


def trace_threads(orc, O, rays, skip, nthreads=None):
    """oracle.trace_bound over chunks of rays on all host cores (the C routine releases the GIL)."""
    import os
    import threading
    n = rays.shape[0]
    out = [np.zeros(n, np.int32), np.zeros(n), np.zeros(n, np.uint8), np.zeros(n)]
    nth = max(1, min(nthreads or os.cpu_count() or 1, n // 256 + 1))
    bounds = np.linspace(0, n, nth + 1).astype(int)

    def work(i):
        a, b = bounds[i], bounds[i + 1]
        if a < b:
            r = orc.trace_bound(O, rays[a:b], skip[a:b])
            for k in range(4):
                out[k][a:b] = r[k]

    ths = [threading.Thread(target=work, args=(i,)) for i in range(nth)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    return out


def tile_mask(cam, tile, tiles):
    """Pixels (flat, row-major) of the tiles [t0, t1) of a W x H tiling, or all pixels."""
    w, h = cam.width, cam.height
    if tiles is None:
        return np.ones(w * h, bool)
    W, H = tile
    ntx = (w + W - 1) // W
    m = np.zeros((h, w), bool)
    for t in range(*tiles):
        tx, ty = t % ntx, t // ntx
        m[ty * H:(ty + 1) * H, tx * W:(tx + 1) * W] = True
    return m.reshape(-1)


def replay_check(cr, orc, S, O, cam, *, max_bounces, mode="direction_reuse", tile=(8, 8), k=None, seed=0, frame=0,
                 tiles=None, nee=False, label="", max_fragile=2e-3, **kw):
    """Render one frame (spp 1) on the GPU with the replay capture and check every stage of
    every bounce against the oracle on the GPU's own inputs:
      trace   the oracle's FP64 closest hit of each captured ray: prim bit-exact unless the
              decision is fragile, t within max(1e-5 t, T_ERR_K terr);
      shade   step b recomputed from trace b-1's captured ray, hit, t and throughput:
              categories, classes, flags, tangent and world exit directions and the next
              throughput bit-exact; spawned origins within spawn_tolerance; with next-event
              estimation the next direction's density within 1e-5 relative;
      radiance the sum of the steps' radiance against the GPU's pixel, 1e-4 relative (1e-6
              absolute below 1e-2), except pixels with a fragile shadow decision.
    Returns (GPU image as float32 (npx, 3), report dict with the measured rates)."""
    from gpu_util import radiance_close
    B = max_bounces
    K = tile[0] * tile[1] if k is None else k
    dbg, bufs = cr.debug_buffers(cam.width, cam.height, B, replay=True)
    img, _ = S.render(cam, spp=1, max_bounces=B, mode=mode, tile=tile, k=K, seed=seed, frame_base=frame, debug=dbg,
                      nee=nee, **kw)
    g = {key: v.cpu().numpy() for key, v in bufs.items()}
    img = img.cpu().numpy().reshape(-1, 3)
    sel = tile_mask(cam, tile, tiles)
    fragile_px = np.zeros(sel.shape, bool)
    n_rays = n_frag = 0
    for b in range(B + 1):
        idx = np.flatnonzero((g["prim"][b] != -2) & sel)
        rays = np.ascontiguousarray(g["ray"][b][idx])
        skip = rays[:, 3].view(np.int32).copy()
        prim, t, fr, terr = trace_threads(orc, O, rays, skip)
        frag = (fr & 1) != 0
        ok = ~frag
        gp, gt = g["prim"][b][idx], g["t"][b][idx].astype(np.float64)
        bad = np.flatnonzero(ok & (gp != prim))
        assert bad.size == 0, f"{label} trace {b}: {bad.size} prim mismatches, e.g. ray {idx[bad[0]]}"
        hit = ok & (prim >= 0)
        terr_ok = np.abs(gt[hit] - t[hit]) <= np.maximum(1e-5 * t[hit], T_ERR_K * terr[hit])
        assert terr_ok.all(), f"{label} trace {b}: {(~terr_ok).sum()} hit distances off"
        n_rays += idx.size
        n_frag += int(frag.sum())
        fragile_px[idx[frag]] = True
    L = np.zeros_like(img, dtype=np.float64)
    staint = np.zeros(sel.shape, bool)
    rkw = dict(max_bounces=B, mode=mode, tile=tile, k=K, seed=seed, frame=frame, nee=nee, tiles=tiles,
               **{key: v for key, v in kw.items() if key in ("hybrid_donor", "nee_shared", "diffuse_roughness",
                                                              "reuse_depth", "interleave")})
    for b in range(1, B + 2):
        r = orc.replay_step(O, cam, b, g["ray"][b - 1], g["prim"][b - 1], g["t"][b - 1], g["beta"][b - 1], **rkw)
        L += r["dL"]
        staint |= r["staint"] != 0
        if b > B:
            continue
        s = sel
        # the GPU's shade visits only groups with a live member: a group with none keeps the
        # capture's prefill (255) as its category where the oracle writes "empty"
        live = g["prim"][b - 1] != -2
        cat_ok = (r["cat"] == g["cat"][b - 1]) | (~live & (g["cat"][b - 1] == 255) & (r["cat"] == 0))
        bad = np.flatnonzero(s & ~cat_ok)
        assert bad.size == 0, f"{label} step {b}: cat differs at {bad.size} pixels, e.g. {bad[0]}"
        bad = np.flatnonzero(s & (r["cls"] != g["cls"][b - 1]))
        assert bad.size == 0, f"{label} step {b}: cls differs at {bad.size} pixels, e.g. {bad[0]}"
        assert np.array_equal(r["flags"][s] & 3, g["flags"][b - 1][s] & 3), f"{label} step {b}: flags"
        for key in ("local", "world"):
            bad = np.flatnonzero(s & (r[key].view(np.uint32) != g[key][b - 1].view(np.uint32)).any(axis=1))
            assert bad.size == 0, f"{label} step {b}: {key} direction differs at {bad.size} pixels"
        traced = g["prim"][b] != -2
        assert np.array_equal(r["next_alive"][s].astype(bool), traced[s]), f"{label} step {b}: alive"
        tr = s & traced
        assert np.array_equal(r["world"][tr].view(np.uint32), g["ray"][b][tr, 4:7].view(np.uint32))
        # throughput: bit-exact, except at GGX points of the rough diffuse class, whose weight
        # pi f is a BRDF evaluation (FP32 on the GPU, FP64 here; ~20 roundings: 1e-5 relative)
        same = (r["next_beta"].view(np.uint32) == g["beta"][b][:, :3].view(np.uint32)).all(axis=1)
        rough = np.zeros(sel.shape, bool)
        tau = kw.get("diffuse_roughness", 0.0)
        if tau > 0:
            src = O.src
            hp = g["prim"][b - 1]
            mat = src.tri_mat[np.maximum(hp, 0)]
            rough = (hp >= 0) & (src.mat_type[mat] == scenes_mat_ggx()) & (src.mat_params[mat, 3] >= tau)
        bad = tr & ~same & ~rough
        assert not bad.any(), f"{label} step {b}: throughput differs at {bad.sum()} pixels"
        rr = tr & rough
        rel = np.abs(r["next_beta"][rr] - g["beta"][b][rr, :3]) / np.maximum(np.abs(r["next_beta"][rr]), 1e-30)
        assert (rel <= 1e-5).all(), f"{label} step {b}: rough-class throughput off by {rel.max()}"
        prev = g["ray"][b - 1][tr]
        tol = spawn_tolerance(prev[:, :3], prev[:, 4:7], g["t"][b - 1][tr], g["ray"][b][tr, :3])
        off = np.abs(r["next_o"][tr] - g["ray"][b][tr, :3]) > tol
        assert not off.any(), f"{label} step {b}: {off.any(axis=1).sum()} spawn points off"
        if nee:
            pr, pg = r["next_pdf"][tr], g["beta"][b][tr, 3].astype(np.float64)
            # GGX's D(h) divides by c^2 (alpha^2 - 1) + 1, which is about alpha^2 at the lobe's
            # peak: FP32 loses log2(1 / alpha^2) bits there, so its density is good to
            # 8 u / alpha^2 (a few roundings of c^2 and of the sum, squared in D)
            src = O.src
            mat = src.tri_mat[np.maximum(g["prim"][b - 1][tr], 0)]
            alpha = np.where(src.mat_type[mat] == scenes_mat_ggx(), src.mat_params[mat, 3], 1.0).astype(np.float64)
            tol = 1e-5 + 8.0 * U / alpha ** 2
            rel = np.abs(pg - pr) / np.maximum(np.abs(pr), 1e-30)
            w = int(np.argmax(rel / tol)) if rel.size else 0
            assert (rel <= tol).all(), (f"{label} step {b}: direction densities off at {(rel > tol).sum()} of "
                                        f"{rel.size}, worst {rel[w]} (alpha {alpha[w]}): gpu {pg[w]} oracle {pr[w]}")
    ok = sel & ~staint
    good, excess, nbad = radiance_close(img, L, ok)
    assert good, f"{label}: {nbad} pixels' radiance off by up to {excess}"
    rep = dict(rays=n_rays, fragile_rays=n_frag, fragile_rate=n_frag / max(1, n_rays),
               pixels=int(sel.sum()), every_stage=float((sel & ~fragile_px & ~staint).sum() / sel.sum()),
               shade_and_radiance=float((sel & ~staint).sum() / sel.sum()))
    print(f"replay {label}: {rep}")
    assert rep["fragile_rate"] <= max_fragile, rep
    return img, rep
