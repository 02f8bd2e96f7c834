"""The error analysis behind the limiter's FP32 screen, checked on the CPU.

The stage kernel lets an element skip the FP64 limiter when an FP32 screen certifies that
Eq. 37-39 give alpha = 1 and that no point of V fails the pressure test of Eq. 47.  The screen
is exact only if its error bounds hold.  This test re-evaluates the screen's arithmetic in
IEEE float32 (numpy; the same operations, constants and order of the bounds, with FMAs where
the kernel writes them). It runs on adversarial 2D P3 elements:
- magnitudes from 1e-20 to 1e20;
- deviations down to 1e-15 of the values;
- one bound per element within 1e-9 .. 1e-2 of an extreme of V, on either side;
- pressure floors near the smallest pressures.
Against the checker's exact limiter, the screen must never certify an element the checker
limits, and it must pass nearly every ordinary element (otherwise it saves nothing).  The
kernel itself is compared with the checker at the same decision boundaries by
tests/test_gpu_limit_screen.py."""
import numpy as np
import pytest

from paper_2407_20966_gb300 import inputs

N, NS, NFP, NV, G = 4, 16, 16, 4, 1.4
f32 = np.float32


def up32(v):
    f = f32(v)
    return np.nextafter(f, f32(np.inf)) if float(f) < v else f


def down32(v):
    f = f32(v)
    return np.nextafter(f, f32(-np.inf)) if float(f) > v else f


def trunc32(xv):
    """FP32 truncation of a double toward zero, 0 below 2^-126, infinite from 2^128."""
    xv = np.asarray(xv, dtype=np.float64)
    with np.errstate(over="ignore"):
        f = xv.astype(f32)
    f = np.where(np.abs(f.astype(np.float64)) > np.abs(xv), np.nextafter(f, f32(0)), f)
    f = np.where(np.abs(xv) < 2.0 ** -126, f32(0), f)
    f = np.where(np.abs(xv) >= 2.0 ** 128, np.copysign(f32(np.inf), xv).astype(f32), f)
    return f.astype(f32)


def fmaf(a, b, c):
    """fmaf with one rounding: the float32 product is exact in float64, the sum p + c is carried
    exactly as s + err (Knuth's two-sum), and s is rounded to float32 with the tie that err
    decides when s falls on a float32 midpoint (the one case where rounding s alone would round
    twice)."""
    p = np.asarray(a, np.float64) * np.asarray(b, np.float64)
    c64 = np.asarray(c, np.float64)
    with np.errstate(invalid="ignore", over="ignore"):
        s = p + c64
        bb = s - p
        err = (p - (s - bb)) + (c64 - bb)
        r = s.astype(f32)
        r64 = r.astype(np.float64)
        other = np.where(s > r64, np.nextafter(r, f32(np.inf)), np.nextafter(r, f32(-np.inf)))
        o64 = other.astype(np.float64)
        mid = (s != r64) & ((r64 + o64) * 0.5 == s)
        take_other = mid & (err != 0) & (np.sign(err) == np.sign(o64 - s))
    return np.where(take_other, other, r).astype(f32)


@pytest.fixture(scope="module")
def consts(orc):
    x, wq = orc.gauss_legendre(N)
    lm = np.array([orc.lagrange(x, j, -1.0) for j in range(N)])
    lp = np.array([orc.lagrange(x, j, 1.0) for j in range(N)])
    wm2 = np.array([wq[k % N] * wq[k // N] for k in range(NS)])
    s2 = 0.0
    for k in range(NS):
        s2 += wm2[k]
    lam = max(np.abs(lm).sum(), np.abs(lp).sum())
    return dict(x=np.asarray(x), wm2=wm2, winv2=1.0 / s2, Wf=wm2.astype(f32), winvf=f32(1.0 / s2),
                lamf=up32(lam), lmf=lm.astype(f32), lpf=lp.astype(f32))


def screen(k, w, bnd, eps, p_floor):
    """The screen's decision for every element: w [NV][E][NS], bnd [2][NV][E]."""
    TINY, CM, CM64 = f32(1e-35), f32((NS + 8) * 2.0 ** -23), f32((2 * NS + 4) * 2.0 ** -53)
    UPF, DNF = f32(1 + 2.0 ** -16), f32(1 - 2.0 ** -20)
    c = w[:, :, 0]
    a = trunc32(w - c[..., None])
    s = np.zeros(c.shape, f32)
    sa = np.zeros(c.shape, f32)
    for n in range(NS):
        s = fmaf(k["Wf"][n], a[..., n], s)
        sa = fmaf(k["Wf"][n], np.abs(a[..., n]), sa)
    amax, amin = a.max(-1), a.min(-1)
    m = (s * k["winvf"]).astype(f32)
    sdev = (a - m[..., None]).astype(f32)
    S = (sa * k["winvf"]).astype(f32)
    C = (np.abs(trunc32(c)) * f32(1 + 2.0 ** -22)).astype(f32)
    em = (CM * S + CM64 * (C + S) + TINY).astype(f32)
    dx, dnn = (amax - m).astype(f32), (amin - m).astype(f32)
    A = np.maximum(amax, -amin)
    fd = np.zeros(c.shape + (NFP,), f32)
    for f in range(4):
        for kk in range(N):
            acc = np.zeros(c.shape, f32)
            for i in range(N):
                l = k["lpf"][i] if f & 1 else k["lmf"][i]
                acc = fmaf(l, sdev[..., kk * N + i if f < 2 else i * N + kk], acc)
            fd[..., f * N + kk] = acc
    fmx, fmn = fd.max(-1), fd.min(-1)
    c32 = trunc32(c)
    M = np.maximum(dx, -dnn)
    enode = (f32(2.0 ** -23) * M + f32(2.0 ** -22) * A + em + TINY).astype(f32)
    eface = (k["lamf"] * (enode + f32((N + 3) * 2.0 ** -24) * M) + (f32(1e-13) * k["lamf"]) * (C + A) + TINY).astype(f32)
    upv = ((np.maximum(dx, fmx) + eface) * UPF).astype(f32)
    dnv = ((np.maximum(-dnn, -fmn) + eface) * UPF).astype(f32)
    need = ((up32(eps) + enode) * UPF).astype(f32)
    hb, lb = trunc32(bnd[1] - c), trunc32(bnd[0] - c)
    with np.errstate(invalid="ignore", over="ignore"):
        ok = ((np.maximum(S, C) <= f32(1e30)) & (dx >= need) & (-dnn >= need) &
              ((hb - m) * DNF >= (upv + f32(2.0 ** -22) * np.abs(hb) + em + TINY) * UPF) &
              ((m - lb) * DNF >= (dnv + f32(2.0 ** -22) * np.abs(lb) + em + TINY) * UPF))
        rl, rh = (m - (dnv + em) * UPF).astype(f32), (m + (upv + em) * UPF).astype(f32)
        bl, bh = (c32 + rl).astype(f32), (c32 + rh).astype(f32)
        sbl = (bl - (f32(2.0 ** -22) * (np.abs(bl) + np.abs(c32)) + f32(2.0 ** -23) * np.abs(rl) + TINY) * UPF).astype(f32)
        sbh = (bh + (f32(2.0 ** -22) * (np.abs(bh) + np.abs(c32)) + f32(2.0 ** -23) * np.abs(rh) + TINY) * UPF).astype(f32)
        fast = ok.all(axis=0)
        rlo = sbl[0]
        mm = np.zeros(rlo.shape, f32)
        for d in (1, 2):
            ad = np.maximum(np.abs(sbl[d]), np.abs(sbh[d]))
            mm = fmaf(ad, ad, mm)
        mm = (mm * f32(1 + 2.0 ** -20)).astype(f32)
        eabs = np.maximum(np.abs(sbl[3]), np.abs(sbh[3]))
        Y = (fmaf(sbl[3], rlo, f32(-0.5) * mm) - f32(1e-6) * fmaf(eabs, rlo, mm)).astype(f32)
        fast &= (rlo > 0) & (down32(G - 1.0) * Y >= f32(2) * up32(p_floor) * rlo + f32(1e-36))
    return fast


def _elements(k, rng, E, amp_range, mag_range):
    base = inputs.random_states(rng, E, 2)
    amp = 10.0 ** rng.uniform(*amp_range, E)
    xi = np.array([k["x"][j % N] for j in range(NS)])
    yi = np.array([k["x"][j // N] for j in range(NS)])
    w = np.empty((NV, E, NS))
    for v in range(NV):
        gx, gy, q = rng.normal(size=(3, E, 1))
        noise = rng.uniform(-1, 1, (E, NS)) * (rng.uniform(size=(E, 1)) < 0.3)
        scale = np.abs(base[:, v:v + 1]) + (0.3 if v in (1, 2) else 0.0)
        w[v] = base[:, v:v + 1] + amp[:, None] * scale * (gx * xi + gy * yi + 0.3 * q * xi * yi + noise)
    w[3] = np.maximum(w[3], 0.5 * (w[1] ** 2 + w[2] ** 2) / w[0] * (1 + 1e-3))
    return w * (10.0 ** rng.uniform(*mag_range, E))[None, :, None]


def _mean_V(orc, k, cfg, om, w):
    V = np.concatenate([w, orc.traces(cfg, om, w)], axis=2)
    return (w * k["wm2"]).sum(axis=2) * k["winv2"], V


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_screen_never_certifies_an_element_the_checker_limits(orc, consts, seed):
    rng = np.random.default_rng(700 + seed)
    mesh = inputs.mesh_2d(32, 32, 0.0, 1.0, 0.0, 1.0, periodic=(True, True))
    om = orc.Mesh(mesh.nbr, mesh.h, mesh.bc)
    E = mesh.n_elem
    screened = near = 0
    for it in range(6):
        w = _elements(consts, rng, E, (-15, -0.7), (-20, 20) if it % 2 else (0, 0))
        eps = [1e-13, 0.0, 1e-9][it % 3]
        cfg = orc.Config(dim=2, p=3, nu=(16, 16), eps=eps)
        mean, V = _mean_V(orc, consts, cfg, om, w)
        dmax, dmin = V.max(axis=2) - mean, V.min(axis=2) - mean
        glo, ghi = 10.0 ** rng.uniform(-2, 0, (2,) + mean.shape)
        cv, cs = rng.integers(0, NV, E), rng.integers(0, 2, E)
        gc = np.where(rng.uniform(size=E) < 0.5, 1.0, -1.0) * 10.0 ** rng.uniform(-9, -2, E)
        for e in range(E):
            (ghi if cs[e] else glo)[cv[e], e] = gc[e]
        bnd = np.stack([mean + dmin * (1 + glo), mean + dmax * (1 + ghi)])
        with np.errstate(invalid="ignore", divide="ignore"):
            P = ((G - 1) * (V[3] - 0.5 * (V[1] ** 2 + V[2] ** 2) / V[0])).min(axis=1)
        cfg.p_floor = float(np.quantile(P[P > 0], 0.02)) * 10.0 ** rng.uniform(-4, 0.05)
        fast = screen(consts, w, bnd, eps, cfg.p_floor)
        _, a = orc.limit(cfg, om, w, bnd)
        assert not (fast & ((a[0] < 1) | (a[1] < 1))).any()
        screened += int(fast.sum())
        near += int(((a[0] < 1) & (a[0] > 1 - 1e-4)).sum())
    assert screened > 100 and near > 500   # both sides of the decision were reached


@pytest.mark.parametrize("amp", [(-8, -6), (-6, -3), (-3, -0.7)])
def test_screen_passes_ordinary_elements(orc, consts, amp):
    """Unit magnitudes, deviations of 1e-8 .. 0.2 of the values, bounds 1e-3 of the deviation
    beyond V, default floors: the screen passes (almost) every element the checker leaves as is."""
    rng = np.random.default_rng(720)
    mesh = inputs.mesh_2d(32, 32, 0.0, 1.0, 0.0, 1.0, periodic=(True, True))
    om = orc.Mesh(mesh.nbr, mesh.h, mesh.bc)
    cfg = orc.Config(dim=2, p=3, nu=(16, 16))
    w = _elements(consts, rng, mesh.n_elem, amp, (0, 0))
    mean, V = _mean_V(orc, consts, cfg, om, w)
    bnd = np.stack([mean + (V.min(axis=2) - mean) * 1.001, mean + (V.max(axis=2) - mean) * 1.001])
    fast = screen(consts, w, bnd, 1e-13, 1e-12)
    _, a = orc.limit(cfg, om, w, bnd)
    keep = (a[0] == 1) & (a[1] == 1)
    assert not (fast & ~keep).any()
    assert fast[keep].mean() > 0.97
