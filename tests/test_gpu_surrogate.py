"""GPU surrogate: BF16 tensor-core gradients against the FP64 oracle, training
on solves of the GPU solver, accuracy against held-out PCG solves, and what
the network gains over the plain method (points answered without a solve)."""
import time

import numpy as np
import pytest

import rve_inputs as ri
from oracle import surrogate as osg

pytestmark = pytest.mark.gpu
TAU = 5e-3          # ensemble-spread gate


@pytest.fixture(scope="module")
def rve():
    import paper_1610_03484_gb300 as pkg
    from paper_1610_03484_gb300 import _build
    _build.build()
    pkg.load_library()
    return pkg


def bf16(a):
    """Round-to-nearest-even to bfloat16, returned as float64."""
    a = np.asarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def oracle_params(buf, member, nparam):
    """Unpack one member from the get_params layout into oracle (W, b) pairs,
    dropping the zero padding (8 of 64 inputs, 33 of 64 outputs)."""
    p = buf[52 + member * nparam: 52 + (member + 1) * nparam]
    dims = [(64, 256), (256, 256), (256, 256), (256, 256), (256, 64)]
    out, o = [], 0
    for l, (k, n) in enumerate(dims):
        W = p[o:o + k * n].reshape(k, n).astype(np.float64)
        o += k * n
        b = p[o:o + n].astype(np.float64)
        o += n
        if l == 0:
            W = W[:8]
        if l == 4:
            W, b = W[:, :33], b[:33]
        out.append((W, b))
    return out


def test_gradients_match_fp64_oracle(rve):
    with rve.Context() as ctx:
        s = rve.Surrogate(ctx, members=1, seed=3)
        rng = np.random.default_rng(0)
        n = 128
        feat = rng.normal(size=(n, 8))
        target = (rng.normal(size=(n, 33)) * 0.5 + 1.0).astype(np.float32)
        g_gpu, loss_gpu = s.gradients(0, feat, target)
        buf = s.get_params()
        nparam = (len(buf) - 52)
        params = oracle_params(buf, 0, nparam)
        # the GPU multiplies BF16 weights and BF16 activations: give the oracle the same weights and inputs
        params_bf = [(bf16(W), b) for W, b in params]
        loss_ref, g_ref = osg.loss_and_grads(params_bf, bf16(feat), target.astype(np.float64), np.ones(33))
        assert abs(loss_gpu - loss_ref) / loss_ref < 1e-2
        g_ref_flat = []
        dims = [(64, 256), (256, 256), (256, 256), (256, 256), (256, 64)]
        for l, ((gW, gb), (k, n_)) in enumerate(zip(g_ref, dims)):
            W = np.zeros((k, n_))
            b = np.zeros(n_)
            W[:gW.shape[0], :gW.shape[1]] = gW
            b[:gb.shape[0]] = gb
            g_ref_flat += [W.ravel(), b]
        g_ref_flat = np.concatenate(g_ref_flat)
        o = 0
        for k, n_ in dims:
            gw = g_gpu[o:o + k * n_]
            rw = g_ref_flat[o:o + k * n_]
            assert np.linalg.norm(gw - rw) / np.linalg.norm(rw) < 2e-2
            o += k * n_
            gb_ = g_gpu[o:o + n_]
            rb = g_ref_flat[o:o + n_]
            assert np.linalg.norm(gb_ - rb) / np.linalg.norm(rb) < 2e-2
            o += n_
        s.free()


@pytest.fixture(scope="module")
def trained(rve):
    grid, p = (6, 6, 4), 1
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    ctx = rve.Context(precision=rve.PREC_MIXED, rtol=1e-7, inner_rtol=1e-6)
    mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
    mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    mesh.set_bc(rve.BC_PERIODIC)
    T, c, t, _, _ = ri.gauss_point_states(1024 + 256, seed=3)
    mid = np.zeros(len(T), np.int32)
    t0 = time.perf_counter()
    Cg, Kg, Dg, st, stats, rc = ctx.macro_update([mesh], T, c, t, mid)
    pcg_s = time.perf_counter() - t0
    assert (st == 0).all()
    feat = ctx.features(mesh, T, c, t)
    s = rve.Surrogate(ctx, members=4, seed=11)
    hist = s.train(feat[:1024], Cg[:1024], Kg[:1024], Dg[:1024], epochs=300, batch=128, lr=2e-3, seed=1)
    yield dict(ctx=ctx, mesh=mesh, s=s, T=T, c=c, t=t, C=Cg, K=Kg, D=Dg, feat=feat, hist=hist, pcg_s=pcg_s)
    s.free()
    mesh.free()
    ctx.close()


def rel(a, b):
    return np.linalg.norm((a - b).reshape(len(a), -1), axis=1) / np.linalg.norm(b.reshape(len(b), -1), axis=1)


def test_training_converges(trained):
    h = trained["hist"]
    assert h[-1] < 0.05 * h[0]


def test_heldout_accuracy_and_spd(trained):
    s, f = trained["s"], trained["feat"][1024:]
    Cp, Kp, Dp, spread = s.predict(f)
    for P, R in ((Cp, trained["C"][1024:]), (Kp, trained["K"][1024:]), (Dp, trained["D"][1024:])):
        assert np.median(rel(P, R)) < 5e-3
        assert np.linalg.eigvalsh(P).min() > 0
    gated = spread <= TAU
    assert gated.mean() > 0.5
    for P, R in ((Cp, trained["C"][1024:]), (Kp, trained["K"][1024:]), (Dp, trained["D"][1024:])):
        assert rel(P[gated], R[gated]).max() < 1e-2


def test_surrogate_with_fallback_gains_over_plain_pcg(rve, trained):
    """What the network gains: held-out points are answered within 1e-2 of
    the PCG solve while only the gated-out points (fewer than half) are
    solved.  On this 6x6x4, p = 1 test mesh a cell solve costs microseconds,
    so the time saved is measured on the benchmark's 24x24x8, p = 2 class
    (bench.py, surrogate leg), not here."""
    ctx, mesh, s = trained["ctx"], trained["mesh"], trained["s"]
    sl = slice(1024, None)
    T, c, t = trained["T"][sl], trained["c"][sl], trained["t"][sl]
    mid = np.zeros(len(T), np.int32)
    Cs, Ks, Ds, st, fb, stats, rc = ctx.macro_update_surrogate([mesh], [s], TAU, T, c, t, mid)
    assert (st == 0).all()
    assert fb.mean() < 0.5
    for P, R in ((Cs, trained["C"][sl]), (Ks, trained["K"][sl]), (Ds, trained["D"][sl])):
        assert rel(P, R).max() < 1e-2
    # fallback points are exact PCG solves
    if fb.any():
        assert rel(Cs[fb == 1], trained["C"][sl][fb == 1]).max() < 1e-6


def test_save_load_round_trip(rve, trained):
    ctx, s = trained["ctx"], trained["s"]
    buf = s.get_params()
    s2 = rve.Surrogate(ctx, members=4, seed=99)
    s2.set_params(buf)
    f = trained["feat"][:64]
    a = s.predict(f)
    b = s2.predict(f)
    # weights round-trip exactly; the saved normalisation scales are FP32
    np.testing.assert_allclose(a[0], b[0], rtol=1e-6)
    np.testing.assert_allclose(a[3], b[3], rtol=1e-6, atol=1e-9)
    s2.free()


# ------------------------------------------------ entry-by-entry against the oracle
DIMS = [(64, 256), (256, 256), (256, 256), (256, 256), (256, 64)]


def unpack_member(buf, member, nparam):
    """One member of the get_params layout as padded (W [in][out], b [out]) pairs."""
    p = buf[52 + member * nparam: 52 + (member + 1) * nparam].astype(np.float64)
    out, o = [], 0
    for k, n in DIMS:
        W = p[o:o + k * n].reshape(k, n)
        o += k * n
        out.append((W, p[o:o + n].copy()))
        o += n
    return out


def flatten(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def emulate_member(params, feat, mean, std):
    """oracle.surrogate.forward layer by layer with the GPU's precision decisions:
    FP32 feature normalisation, BF16 weights and BF16 activations between
    layers (FP32 accumulation is replaced by the oracle's FP64)."""
    inv = (np.float32(1.0) / std.astype(np.float32))
    x = bf16((feat.astype(np.float32) - mean.astype(np.float32)) * inv)
    h = np.zeros((len(feat), 64))
    h[:, :8] = x
    for l, (W, b) in enumerate(params):
        a, _ = osg.forward([(bf16(W), b)], h)
        h = bf16(osg.silu(a)) if l < len(params) - 1 else a
    return h[:, :33]


def test_predict_matches_oracle_entry_by_entry(rve, trained):
    """Inference (features, four BF16 members, softplus head, L L^T, ensemble mean
    and spread) against oracle.surrogate.forward -> factor_entries ->
    tensors_from_factors on the same BF16-rounded weights and inputs.  Tolerance
    of a BF16 network: an activation whose FP32 and FP64 sums round to different
    BF16 neighbours moves a member's tensors by about 5e-4."""
    s = trained["s"]
    f = trained["feat"][1024:1024 + 128]
    Cg, Kg, Dg, spread_g = s.predict(f)
    buf = s.get_params()
    members = 4
    nparam = (len(buf) - 52) // members
    mean, std, ref = buf[:8], buf[8:16], buf[49:52].astype(np.float64)
    Ts = []
    for e in range(members):
        z = emulate_member(unpack_member(buf, e, nparam), f, mean, std)
        Ts.append(osg.tensors_from_factors(osg.factor_entries(z)))
    Tm = [np.mean([T[b] for T in Ts], axis=0) for b in range(3)]
    for b, (G, r) in enumerate(((Cg, ref[0]), (Kg, ref[1]), (Dg, ref[2]))):
        err = rel(G, Tm[b] * r)
        assert err.max() < 2e-3, (b, err.max())
    spread = np.zeros(len(f))
    for b in range(3):
        den = np.linalg.norm(Tm[b].reshape(len(f), -1), axis=1)
        for T in Ts:
            spread = np.maximum(spread, np.linalg.norm((T[b] - Tm[b]).reshape(len(f), -1), axis=1) / den)
    assert np.abs(spread_g - spread).max() < 2e-3, np.abs(spread_g - spread).max()


def test_adam_steps_match_oracle(rve):
    """Two steps of the GPU's minibatch Adam (one batch per epoch, learning rate
    lr then 0.51 lr from the cosine schedule) against oracle.surrogate.adam_step
    fed with the GPU's own gradients at the same weights: FP32 agreement.  The
    first step must be -lr * g / (|g| + eps) (the bias-corrected first step)."""
    rng = np.random.default_rng(21)
    n, lr = 64, 1e-3
    feat = rng.normal(size=(n, 8)) * [10, 0.4, 1, 1e9, 4e9, 1e9, 5e8, 0.05] + [40, 0.75, 2, 3e9, 45e9, 12e9, 5e9, 0.2]
    A = rng.normal(size=(n, 6, 6))
    Cc = A @ np.swapaxes(A, 1, 2) + 6 * np.eye(6)
    B3 = rng.normal(size=(n, 3, 3))
    Kk = B3 @ np.swapaxes(B3, 1, 2) + 3 * np.eye(3)
    Dd = 2 * Kk + np.eye(3)
    with rve.Context() as ctx:
        s0 = rve.Surrogate(ctx, members=1, seed=5)
        buf0 = s0.get_params()
        s1 = rve.Surrogate(ctx, members=1, seed=5)
        s1.train(feat, Cc, Kk, Dd, epochs=1, batch=n, lr=lr, seed=1)
        buf1 = s1.get_params()
        s2 = rve.Surrogate(ctx, members=1, seed=5)
        s2.train(feat, Cc, Kk, Dd, epochs=2, batch=n, lr=lr, seed=1)
        buf2 = s2.get_params()
        header = buf2[:52]
        assert np.array_equal(header, buf1[:52])
        ref = header[49:52].astype(np.float64)
        sym = lambda T: 0.5 * (T + np.swapaxes(T, 1, 2))
        target = osg.factors_from_tensors(sym(Cc) / ref[0], sym(Kk) / ref[1], sym(Dd) / ref[2]).astype(np.float32)
        grads = []
        for pb in (buf0, buf1):
            sg = rve.Surrogate(ctx, members=1, seed=5)
            sg.set_params(np.concatenate([header, pb[52:]]).astype(np.float32))
            g, _ = sg.gradients(0, feat, target)
            grads.append(g.astype(np.float64))
            sg.free()
        for x in (s0, s1, s2):
            x.free()
    nparam = len(buf0) - 52
    P0 = unpack_member(buf0, 0, nparam)
    state = [(np.zeros_like(W), np.zeros_like(W), np.zeros_like(b), np.zeros_like(b)) for W, b in P0]

    def as_pairs(flat):
        out, o = [], 0
        for k, nn in DIMS:
            out.append((flat[o:o + k * nn].reshape(k, nn), flat[o + k * nn:o + k * nn + nn]))
            o += k * nn + nn
        return out

    P1 = osg.adam_step(P0, as_pairs(grads[0]), state, lr, 1)
    P2 = osg.adam_step(P1, as_pairs(grads[1]), state, 0.51 * lr, 2)
    f0, f1, f2 = flatten(P0), flatten(P1), flatten(P2)
    g1 = grads[0]
    # first step identity on the oracle side (documents what is compared)
    np.testing.assert_allclose(f1 - f0, -lr * g1 / (np.abs(g1) + 1e-8), rtol=1e-12, atol=1e-15)
    gpu1 = buf1[52:].astype(np.float64)
    gpu2 = buf2[52:].astype(np.float64)
    ulp = np.spacing(np.abs(f0).astype(np.float32)).astype(np.float64)
    # The trainer shuffles the batch rows, so its batch sums run in another order
    # than the gradient recomputed here (FP32, about 1e-7 of the summed terms).
    # Adam maps g to -lr g / (|g| + eps): where |g| >> eps the step does not depend
    # on that rounding; near |g| ~ eps (or a sign change) it does, so those
    # entries are only bounded by the step size.
    g2 = grads[1]
    big1 = np.abs(g1) > 1e-5
    big = big1 & (np.abs(g2) > 1e-5)
    assert big.mean() > 0.5
    d1 = np.abs(gpu1 - f1)
    assert (d1[big1] <= 4 * ulp[big1] + 1e-5 * lr).all(), d1[big1].max()
    assert (np.abs(gpu1 - f0) <= lr + 4 * ulp).all()
    d2 = np.abs(gpu2 - f2)
    assert (d2[big] <= 8 * ulp[big] + 1e-4 * lr).mean() > 0.999, np.sort(d2[big])[-10:]
    assert d2[big].max() < 0.05 * lr, d2[big].max()
    assert (np.abs(gpu2 - f0) <= 2.1 * lr + 8 * ulp).all()


def test_surrogate_gain_on_bench_class(rve):
    """The trained weights of the benchmark's class (24x24x8, p = 2) answer 2048
    Gauss points, with spread-gated fallback, faster than plain batched PCG
    solves them, within 1e-2 of the PCG tensors."""
    import os
    import bench
    if not os.path.exists(bench.SURROGATE_FILE):
        pytest.skip("no trained weights")
    z = np.load(bench.SURROGATE_FILE)
    xyz, tets, phase, tangent = ri.weave_rve(24, 24, 8)
    T, c, t, _, _ = ri.gauss_point_states(2048 + 512, 41)
    with rve.Context(precision=rve.PREC_MIXED, rtol=bench.RTOL, inner_rtol=bench.INNER_RTOL, max_refine=4) as ctx:
        mesh = ctx.mesh_load(xyz, tets, 2, phase, tangent)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        mesh.set_bc(rve.BC_PERIODIC)
        s = rve.Surrogate(ctx, members=int(z["members"]), seed=0)
        s.set_params(z["params"])
        mid = np.zeros(2048, np.int32)
        w = slice(2048, None)   # warm-up on other points
        ctx.macro_update_surrogate([mesh], [s], bench.SURROGATE_TAU, T[w], c[w], t[w], mid[:512])
        ctx.macro_update([mesh], T[w][:64], c[w][:64], t[w][:64], mid[:64])
        t0 = time.perf_counter()
        Cs, Ks, Ds, st, fb, _, _ = ctx.macro_update_surrogate([mesh], [s], bench.SURROGATE_TAU, T[:2048], c[:2048],
                                                              t[:2048], mid)
        sur_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        Cp, Kp, Dp, stp, _, _ = ctx.macro_update([mesh], T[:2048], c[:2048], t[:2048], mid)
        pcg_s = time.perf_counter() - t0
        s.free()
        mesh.free()
    assert (st == 0).all() and (stp == 0).all()
    for P, R in ((Cs, Cp), (Ks, Kp), (Ds, Dp)):
        assert rel(P, R).max() < 1e-2
    assert sur_s < 0.5 * pcg_s, (sur_s, pcg_s, fb.mean())


def test_fused_inference_matches_layer_by_layer(rve, trained):
    """The fused whole-network kernel against one tensor-core GEMM per member and
    layer: the same BF16 products in the same order, so the same tensors up to the
    last bits of the FP32 head.  Sizes: a ragged 1 000-point set (a partial 128-row
    tile, M = 1024 padded) and 64 points (a single 64-row tile)."""
    s = trained["s"]
    for n in (1000, 64):
        f = trained["feat"][:n]
        s.set_fused(True)
        a = s.predict(f)
        s.set_fused(False)
        b = s.predict(f)
        s.set_fused(True)
        for x, y in zip(a, b):
            np.testing.assert_allclose(x, y, rtol=1e-6, atol=1e-12 * np.abs(y).max())
