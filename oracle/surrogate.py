"""Plain numpy oracle of the learned surrogate's layers (FP64).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` may use it.  It shares no code with the CUDA
library.  The paper has no learned component; each function below states the
definition it writes out.

Tensors are channels-last volumes [batch][n2][n1][n0][C], periodic in the
three spatial axes.  A 3x3x3 layer has weights W[co][tap][ci] with
tap = (dz*3 + dy)*3 + dx and spatial offset (dz-1, dy-1, dx-1).

Where the tensor-core path rounds to bfloat16 (its operands), the oracle
rounds the same values the same way (``bf16``) and then computes in FP64, so
the only difference left is the order and precision of the accumulation.
"""
import numpy as np

TAPS = [(dz - 1, dy - 1, dx - 1) for dz in range(3) for dy in range(3) for dx in range(3)]


def bf16(x):
    """Round to bfloat16 as the device does: to binary32 (nearest), then to the
    8-bit significand of bfloat16 (nearest, ties to even).  Returns FP64."""
    u = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits(x):
    """The uint16 bit patterns of bf16(x)."""
    return (bf16(x).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


def from_bf16_bits(b):
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def shift(x, off):
    """s[p] = x[p + off] on the periodic box (axes 1, 2, 3 are z, y, x)."""
    return np.roll(x, shift=(-off[0], -off[1], -off[2]), axis=(1, 2, 3))


def conv3(x, W, b=None, relu=False):
    """Cross-correlation y[p][co] = b[co] + sum_{tap, ci} x[p + off(tap)][ci] W[co][tap][ci],
    then max(0, .) if relu."""
    y = np.zeros(x.shape[:4] + (W.shape[0],))
    for tap, off in enumerate(TAPS):
        y += np.einsum("bzyxc,oc->bzyxo", shift(x, off), W[:, tap, :])
    if b is not None:
        y += b
    return np.maximum(y, 0.0) if relu else y


def conv3_input_grad(gy, W, mask=None):
    """Adjoint of conv3 in x: gx[q][ci] = sum_{tap, co} gy[q - off(tap)][co] W[co][tap][ci],
    zeroed where mask <= 0 (the ReLU derivative of the layer below)."""
    gx = np.zeros(gy.shape[:4] + (W.shape[2],))
    for tap, off in enumerate(TAPS):
        gx += np.einsum("bzyxo,oc->bzyxc", shift(gy, (-off[0], -off[1], -off[2])), W[:, tap, :])
    return gx if mask is None else np.where(mask > 0, gx, 0.0)


def conv3_weight_grad(x, gy):
    """gW[co][tap][ci] = sum_p gy[p][co] x[p + off(tap)][ci];  gb[co] = sum_p gy[p][co]."""
    gW = np.stack([np.einsum("bzyxo,bzyxc->oc", gy, shift(x, off)) for off in TAPS], axis=1)
    return gW, gy.sum(axis=(0, 1, 2, 3))


def adam(w, g, m, v, lr, b1, b2, eps, t):
    """One step of Adam (Kingma & Ba 2015, Algorithm 1), t >= 1; returns (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def mse(y, t):
    """loss = mean (y - t)^2 over points and channels; gradient 2 (y - t) / count."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


# ---------------------------------------------------------------- the surrogate
#
# One call replaces four RK4 steps of the method (Delta = 4 dt) on a periodic
# global patch of spacing h.  L is the method's 4th-order centred Laplacian.
# The state advances by the fourth-order Taylor step of the semi-discrete wave
# equation (d psi/dt = Pi, d Pi/dt = L psi; for this linear system one RK4
# step of size Delta) plus the network's learned remainder; the network sees
# the state and its Laplacians scaled to order one.  The
# operation order below is the order in which every value is defined (the
# device computes the same FP64 operations, each rounded once).

LAYERS = [(7, 32, True), (32, 32, True), (32, 32, True), (32, 2, False)]  # (cin, cout, relu)
PADDED = [(8, 32), (32, 32), (32, 32), (32, 8)]                            # stored channel counts


def param_count():
    return sum(co * 27 * ci + co for ci, co in PADDED)


def unpack_params(flat):
    """Flat padded binary32 layout -> [(W[co][27][ci], b[co])] with the real channel counts."""
    out, off = [], 0
    for (ci, co, _), (pci, pco) in zip(LAYERS, PADDED):
        W = np.asarray(flat[off:off + pco * 27 * pci], dtype=np.float64).reshape(pco, 27, pci)
        off += pco * 27 * pci
        b = np.asarray(flat[off:off + pco], dtype=np.float64)
        off += pco
        out.append((W[:co, :, :ci].copy(), b[:co].copy()))
    return out


def pack_params(layers, dtype=np.float32):
    parts = []
    for (W, b), (pci, pco) in zip(layers, PADDED):
        Wp = np.zeros((pco, 27, pci))
        Wp[:W.shape[0], :, :W.shape[2]] = W
        bp = np.zeros(pco)
        bp[:b.shape[0]] = b
        parts += [Wp.ravel(), bp]
    return np.concatenate(parts).astype(dtype)


def coefficients(dt, h):
    """Delta, Delta^2/2, Delta^3/6, Delta^4/24, 1/(12 h^2) and the powers Delta^1..6."""
    D = 4.0 * dt
    powers = [D, D * D, D * D * D, D * D * D * D, D * D * D * D * D, D * D * D * D * D * D]
    return D, D * D / 2.0, D * D * D / 6.0, D * D * D * D / 24.0, 1.0 / (12.0 * h * h), powers


def lap4(u, h):
    """4th-order centred Laplacian on the periodic box, u[batch][z][y][x]:
    per axis (16 (u[-1] + u[1]) - (u[-2] + u[2])) - 30 u, summed x, y, z,
    times 1 / (12 h^2)."""
    inv = 1.0 / (12.0 * h * h)
    S = []
    for ax in (3, 2, 1):
        m1, p1 = np.roll(u, 1, axis=ax), np.roll(u, -1, axis=ax)
        m2, p2 = np.roll(u, 2, axis=ax), np.roll(u, -2, axis=ax)
        S.append((16.0 * (m1 + p1) - (m2 + p2)) - 30.0 * u)
    return ((S[0] + S[1]) + S[2]) * inv


def scales(psi, pi, dt):
    """Per sample s = 1 / max(|psi|, Delta |Pi|), the maximum and the quotient
    each rounded to binary32 (1 for a zero state)."""
    D = 4.0 * dt
    m = np.maximum(np.abs(psi), D * np.abs(pi)).reshape(psi.shape[0], -1).max(axis=1).astype(np.float32)
    return np.where(m > 0, (1.0 / np.maximum(m.astype(np.float64), 1e-300)).astype(np.float32), np.float32(1.0))


def features(psi, pi, dt, h):
    """x = bf16(s psi, s D Pi, s D^2 L psi, s D^3 L Pi, s D^4 L^2 psi, s D^5 L^2 Pi,
    s D^6 L^3 psi) (D = Delta: the terms of the Taylor series of the evolution,
    each scaled to order one) and s."""
    Dk = coefficients(dt, h)[5]
    s = scales(psi, pi, dt).astype(np.float64)[:, None, None, None]
    lp, lq = lap4(psi, h), lap4(pi, h)
    llp, llq = lap4(lp, h), lap4(lq, h)
    lllp = lap4(llp, h)
    f = [s * psi, (s * Dk[0]) * pi, (s * Dk[1]) * lp, (s * Dk[2]) * lq, (s * Dk[3]) * llp, (s * Dk[4]) * llq,
         (s * Dk[5]) * lllp]
    return bf16(np.stack(f, axis=-1)), s[:, 0, 0, 0].astype(np.float32)


def targets(psi0, pi0, psi1, pi1, s, dt, h, sigma):
    """The remainder of the method's four steps over the Taylor step, scaled."""
    D, hD2, D36, D424, _, _ = coefficients(dt, h)
    lp, lq = lap4(psi0, h), lap4(pi0, h)
    llp, llq = lap4(lp, h), lap4(lq, h)
    r0 = ((((psi1 - psi0) - D * pi0) - hD2 * lp) - D36 * lq) - D424 * llp
    r1 = ((((pi1 - pi0) - D * lp) - hD2 * lq) - D36 * llp) - D424 * llq
    cs = np.asarray(s, np.float64)[:, None, None, None] / sigma
    return np.stack([(cs * r0).astype(np.float32), ((cs * D) * r1).astype(np.float32)], axis=-1).astype(np.float64)


def apply(psi0, pi0, s, y, dt, h, sigma):
    """(psi1, Pi1) from the Taylor step and the network output y[..., 0:2]."""
    D, hD2, D36, D424, _, _ = coefficients(dt, h)
    lp, lq = lap4(psi0, h), lap4(pi0, h)
    llp, llq = lap4(lp, h), lap4(lq, h)
    a = sigma / np.asarray(s, np.float64)[:, None, None, None]
    psi1 = ((((psi0 + D * pi0) + hD2 * lp) + D36 * lq) + D424 * llp) + a * y[..., 0]
    pi1 = ((((pi0 + D * lp) + hD2 * lq) + D36 * llp) + D424 * llq) + (a / D) * y[..., 1]
    return psi1, pi1


def net_forward(x, params, rounded=True):
    """Activations [x, a1, a2, a3] and the FP64 output y.  rounded: the
    hidden activations are stored in bfloat16, as the device stores them."""
    layers = unpack_params(params)
    acts = [x]
    a = x
    for l, ((W, b), (_, _, relu)) in enumerate(zip(layers, LAYERS)):
        Wr = bf16(W) if rounded else W
        br = b.astype(np.float32).astype(np.float64) if rounded else b
        z = conv3(a, Wr, br, relu=relu)
        if l < len(LAYERS) - 1:
            a = bf16(z) if rounded else z
            acts.append(a)
        else:
            return acts, z


def net_grads(x, params, t, rounded=True):
    """Loss and d loss / d params (flat padded layout) of the mean squared error
    of the network output against t; gradients at layer outputs are stored in
    bfloat16 where the device stores them (rounded)."""
    layers = unpack_params(params)
    acts, y = net_forward(x, params, rounded)
    loss, g = mse(y, t)
    g = bf16(g) if rounded else g
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        grads[l] = conv3_weight_grad(acts[l], g)
        if l == 0:
            break
        W = bf16(layers[l][0]) if rounded else layers[l][0]
        g = conv3_input_grad(g, W, mask=acts[l])
        g = bf16(g) if rounded else g
    return loss, pack_params(grads, np.float64)


def residual(psi0, pi0, psi1, pi1, dt, h):
    """Per sample max(|R_psi|, Delta |R_Pi|) and max(|psi0|, Delta |Pi0|), with the
    two-point quadrature with end corrections of d psi/dt = Pi, d Pi/dt = L psi:
    R_psi = psi1 - psi0 - D/2 (Pi0 + Pi1) + D^2/12 (L psi1 - L psi0),
    R_Pi  = Pi1 - Pi0 - D/2 (L psi0 + L psi1) + D^2/12 (L Pi1 - L Pi0)."""
    D = 4.0 * dt
    lp0, lq0, lp1, lq1 = (lap4(u, h) for u in (psi0, pi0, psi1, pi1))
    rp = (psi1 - psi0) - D / 2 * (pi0 + pi1) + D * D / 12 * (lp1 - lp0)
    rq = (pi1 - pi0) - D / 2 * (lp0 + lp1) + D * D / 12 * (lq1 - lq0)
    B = psi0.shape[0]
    r = np.maximum(np.abs(rp), D * np.abs(rq)).reshape(B, -1).max(axis=1)
    m = np.maximum(np.abs(psi0), D * np.abs(pi0)).reshape(B, -1).max(axis=1)
    return r, m


def hermite5(tau):
    """Quintic Hermite basis on [0, 1]: weights of y0, y0', y0'', y1, y1', y1''
    (derivatives in units of the interval)."""
    t = tau
    return np.array([1 - 10 * t**3 + 15 * t**4 - 6 * t**5, t - 6 * t**3 + 8 * t**4 - 3 * t**5,
                     0.5 * (t**2 - 3 * t**3 + 3 * t**4 - t**5), 10 * t**3 - 15 * t**4 + 6 * t**5,
                     -4 * t**3 + 7 * t**4 - 3 * t**5, 0.5 * (t**3 - 2 * t**4 + t**5)])


# ---------------------------------------------------------------------------
# The hybrid call with local patches (mpw_step_surrogate): the surrogate
# advances the periodic global patch four steps at once while the local
# patches take the method's four RK4 steps.  An extension of the paper's
# method, laid out here from its definition, over the C oracle's pieces.

def hermite_stage_weights(m, l):
    """Weights of (y0, y0', y0'', y1, y1', y1'') (derivatives in units of the
    call's interval Delta = 4 dt) that give the RK4 stage state of substage l
    of step m of a call.  For the linear system y' = A y the RK4 stage states
    of a step that starts from u are u, u + dt/2 u', u + dt/2 u' + dt^2/4 u'',
    u + dt u' + dt^2/2 u'' + dt^3/4 u''' (each stage input is u plus dt times
    the previous stage's slope); u and its time derivatives are those of the
    quintic Hermite interpolant at tau = m / 4, with d/dt = (1 / Delta) d/dtau
    and dt / Delta = 1/4."""
    tau = m / 4.0
    stage = [(1.0, 0.0, 0.0, 0.0), (1.0, 0.5, 0.0, 0.0), (1.0, 0.5, 0.25, 0.0), (1.0, 1.0, 0.5, 0.25)][l]
    t = np.polynomial.Polynomial([0.0, 1.0])
    basis = [1 - 10 * t**3 + 15 * t**4 - 6 * t**5, t - 6 * t**3 + 8 * t**4 - 3 * t**5,
             0.5 * (t**2 - 3 * t**3 + 3 * t**4 - t**5), 10 * t**3 - 15 * t**4 + 6 * t**5,
             -4 * t**3 + 7 * t**4 - 3 * t**5, 0.5 * (t**3 - 2 * t**4 + t**5)]
    w = np.zeros(6)
    for k, ck in enumerate(stage):
        if ck == 0.0:
            continue
        for j, b in enumerate(basis):
            # dt^k d^k/dt^k = (1/4)^k d^k/dtau^k
            w[j] += ck * 0.25**k * b.deriv(k)(tau) if k else ck * b(tau)
    return w


def hybrid_call(o, params, dt, h, sigma, P=6):
    """One hybrid call on the oracle simulation o (global patch 0 periodic,
    local patches 1..): from the state at t, with the flags at t (and the
    revival they bring), the global's covered cells refilled from the local
    patches (Local-to-Global) and its dead cells interpolated from them, the
    surrogate's global state four steps later (features, network, update);
    the local patches then take four RK4 steps of the method whose
    Global-to-Local data come from the global stage states of the quintic
    Hermite interpolant between the two global states; the global ends at the
    surrogate's state.  params: the network's flat parameters (None: the
    network off, the fourth-order Taylor step alone)."""
    from oracle import pyoracle as po
    t = o.time
    ng = po.NG
    o.compute_flags()
    o.fill_ghosts(t)
    o.fill_dead(t)
    ps, pq = o.get_padded(0, which=1)
    inner = (slice(ng, -ng),) * 3
    psi0, pi0 = ps[inner][None].copy(), pq[inner][None].copy()
    x, s = features(psi0, pi0, dt, h)
    y = np.zeros(psi0.shape + (8,)) if params is None else net_forward(x, params)[1]
    psi1, pi1 = apply(psi0, pi0, s, y, dt, h, sigma)
    D = 4.0 * dt
    lp0, lq0, lp1, lq1 = lap4(psi0, h), lap4(pi0, h), lap4(psi1, h), lap4(pi1, h)
    # interpolant data per field, derivatives in units of the interval
    data_psi = (psi0, D * pi0, D * D * lp0, psi1, D * pi1, D * D * lp1)
    data_pi = (pi0, D * lp0, D * D * lq0, pi1, D * lp1, D * D * lq1)
    for m in range(4):
        stages = []
        for l in range(4):
            w = hermite_stage_weights(m, l)
            stages.append((sum(wj * v for wj, v in zip(w, data_psi))[0], sum(wj * v for wj, v in zip(w, data_pi))[0]))
        o.step_locals(dt, stages)
    o.set_fields(0, psi1[0], pi1[0])
    return psi1[0], pi1[0]
