"""Oracle of the volume-of-fluid step (test infrastructure only): MTHINC reconstruction and
directional-split advection of the volume fraction, FP64, triply periodic, uniform spacing per
direction.

Paper (arXiv 2204.08834): Sec. 3.1 (the volume fraction phi, the MTHINC indicator H of
Eq. h_parameter, the split update Eq. phi_split and the divergence correction
Eq. vof_corr_step) and Appendix A (the reconstruction polynomial T, Eqs. qud_fun, q1_comp,
q2_comp, l_comp; normals and curvature from Youngs' corner gradients, Eqs. normal and kappa_t;
the normalisation d_th, Eqs. int and int_x/int_y/int_z; the numerical fluxes, Eqs. fx/fy/fz
and their swept-interval form; the overall VoF algorithm).

H(x~) = (1 + tanh(beta (T(x~) + d))) / 2 in the cell's local coordinates x~ in [0, 1]^3.

Readings of what the paper leaves open or prints garbled (V1-V10):
  V1  Local coordinates x~ = (x - x_{i-1/2}) / dx (likewise y, z): the cell is [0, 1]^3 with
      centre (1/2, 1/2, 1/2), where grad T = n and grad grad T = K are imposed.
  V2  Gradients are taken in cell units (d/dx~).  The tensor that enters T is K = grad n, the
      one that makes grad T = n and grad grad T = K consistent (the paper's K = -grad n fixes
      the sign of its curvature kappa = -tr K; here kappa = -tr grad n = -div n); K is
      symmetrised.
  V3  Flags: with p the direction of exact integration, c = (1, 1, 1) - e_p; the quadratic term
      of direction a is kept iff c_a = 1, the cross term of a and b iff c_a c_b = 1, so T is
      linear in x~_p (case 1: c = [0,1,1]; case 2: [1,0,1]; case 3: [1,1,0], where the printed
      case-3 flags are garbled).  Then L_a = n_a - (c_a / 2)(K_aa + sum_{b != a} c_b K_ab).
  V4  The two-point Gauss-Legendre rule on [0, 1]: nodes (1 -+ 1/sqrt 3)/2, weights 1/2 (the
      printed "1 + sqrt 3/2 [...]" is garbled); on a sub-interval [lo, hi] the nodes map
      linearly and the weights are (hi - lo)/2.
  V5  d_th is the root of the volume equation: the integral of H over the cell, exact along p
      (the antiderivative in log cosh) and Gauss along the other two directions, equals phi.
      The equation is increasing in d; the root is found here by bisection.  The paper's quartic
      in D = exp(2 beta d_th) has D as its positive root, with coefficients
      alpha_k = e_k(G) (A^k - A^2 Q), e_k the elementary symmetric polynomials of the four
      G_q = exp(2 beta g_q) (g_q: T at x~_p = 0 and the Gauss node q), A = exp(2 beta a_L^p),
      Q = exp(4 beta a_L^p (2 phi - 1)); the printed alpha_2 is garbled (its e_2 is
      B-B+ + C-C+ + (B- + B+)(C- + C+)).
  V6  Fluxes: the flux through a face is the integral of H of the upwind cell over the box swept
      in dt: along the split direction the fraction |u| dt / dl at the cell's downwind side
      ([1 - c, 1] for u >= 0, [0, -c] for u < 0, c = u dt / dl), [0, 1] along the other two;
      the same quadrature as V5 (exact along the upwind cell's p over its interval, Gauss over
      the others).  The printed prefactor Delta x~ is the interval length that the Gauss
      weights carry.  F is a fraction of the cell volume, the f/dl of Eq. phi_split.
  V7  Case: p = x if |n_x| >= |n_y| and |n_x| >= |n_z|, else p = y if |n_y| >= |n_z|, else z,
      decided on the components of the Youngs gradient m (n = m / |m|, the same comparisons).
      The paper states no precision; this integer decision (and the zero-gradient test of V8)
      is taken in binary32 arithmetic, the precision of the GPU kernel, with the operations of
      youngs() in the same order (youngs_m32), so that both sides decide alike.  n, K and T
      stay binary64.
  V8  A cell with phi <= eps or phi >= 1 - eps (eps = 1e-8), or with a zero Youngs gradient,
      is uniform: H = phi on the whole cell.
  V9  The splits run in the fixed order x, y, z; n, K and d_th are recomputed from phi^x before
      the y split and from phi^y before the z split; phi is not clipped.
  V10 Triply periodic domain; the face velocity u[k][j][i] sits on the x face i+1/2 (v, w
      likewise), as in the projection step.

Arrays are (nz, ny, nx), x fastest.  Direction index a = 0, 1, 2 for x, y, z (numpy axis 2 - a).
"""

import numpy as np

EPS_PURE = 1e-8
GAUSS = ((1.0 - 1.0 / np.sqrt(3.0)) / 2.0, (1.0 + 1.0 / np.sqrt(3.0)) / 2.0)


def axis(a):
    """numpy axis of direction a (0: x, 1: y, 2: z)."""
    return 2 - a


def sh(f, d, a):
    """f shifted along direction a so that sh(f, +1, a)[i] = f[i + 1] (periodic)."""
    return np.roll(f, -d, axis=axis(a))


# ------------------------------------------------------- normals and curvature (App. A.1.1)

def youngs(phi):
    """Youngs' gradients (V2): at every cell corner (i+1/2, j+1/2, k+1/2), stored at the cell
    (i, j, k) below it, the difference across the corner averaged over the four cell pairs;
    the cell gradient m is the average of its eight corner gradients, the cell normal
    n = m / |m|; K_ab = d n_b / d x~_a from the normalised corner gradients differenced across
    the cell (averaged over the four corner pairs), symmetrised.  Returns (m, n, K) with
    m, n lists of 3 arrays and K a dict {(a, b): array} for a <= b."""
    mc = []
    for a in range(3):
        d = sh(phi, 1, a) - phi                      # across the corner along a
        o1, o2 = [b for b in range(3) if b != a]
        mc.append(0.25 * (d + sh(d, 1, o1) + sh(d, 1, o2) + sh(sh(d, 1, o1), 1, o2)))
    # cell gradient: the 8 corners of cell i are the corner cells i-1, i along each direction
    m = []
    for a in range(3):
        s = mc[a]
        for b in range(3):
            s = s + sh(s, -1, b)
        m.append(s / 8.0)
    mm = np.sqrt(m[0] ** 2 + m[1] ** 2 + m[2] ** 2)
    safe = np.where(mm > 0.0, mm, 1.0)
    n = [np.where(mm > 0.0, m[a] / safe, 0.0) for a in range(3)]
    cm = np.sqrt(mc[0] ** 2 + mc[1] ** 2 + mc[2] ** 2)
    csafe = np.where(cm > 0.0, cm, 1.0)
    nc = [np.where(cm > 0.0, mc[a] / csafe, 0.0) for a in range(3)]
    dn = {}
    for a in range(3):                               # d/dx~_a across the cell
        o1, o2 = [b for b in range(3) if b != a]
        for b in range(3):
            d = nc[b] - sh(nc[b], -1, a)             # corner at the cell's upper a side minus lower
            d = d + sh(d, -1, o1)
            d = d + sh(d, -1, o2)
            dn[(a, b)] = d / 4.0
    K = {}
    for a in range(3):
        for b in range(a, 3):
            K[(a, b)] = 0.5 * (dn[(a, b)] + dn[(b, a)])
    return m, n, K


def youngs_m32(phi):
    """The cell gradient m of youngs() in binary32 arithmetic, the same operations in the same
    order (phi rounded to binary32 first): the input of the case decision (V7)."""
    f = phi.astype(np.float32)
    q = np.float32(0.25)
    mc = []
    for a in range(3):
        d = sh(f, 1, a) - f
        o1, o2 = [b for b in range(3) if b != a]
        mc.append(q * (((d + sh(d, 1, o1)) + sh(d, 1, o2)) + sh(sh(d, 1, o1), 1, o2)))
    m = []
    for a in range(3):
        s = mc[a]
        for b in range(3):
            s = s + sh(s, -1, b)
        m.append(s * np.float32(0.125))
    return m


def curvature(phi):
    """kappa = -tr K = -div n (V2), in cell units."""
    _, _, K = youngs(phi)
    return -(K[(0, 0)] + K[(1, 1)] + K[(2, 2)])


# ------------------------------------------------------ reconstruction polynomial (App. A.1)

def polynomial(n, K, m=None):
    """Case p (V7, on the gradient m when given, else on n) and the coefficients of T
    (Eqs. qud_fun, q1_comp, q2_comp, l_comp with the flags of V3):
    T = sum_a q_a x~_a^2 + sum_{a<b} r_ab x~_a x~_b + sum_a L_a x~_a.
    Returns (p, q[3], r{(a,b)}, L[3])."""
    v = n if m is None else m
    ax_, ay_, az_ = np.abs(v[0]), np.abs(v[1]), np.abs(v[2])
    p = np.where((ax_ >= ay_) & (ax_ >= az_), 0, np.where(ay_ >= az_, 1, 2))
    c = [(p != a).astype(np.float64) for a in range(3)]
    q = [c[a] * 0.5 * K[(a, a)] for a in range(3)]
    r = {(a, b): c[a] * c[b] * K[(a, b)] for a in range(3) for b in range(a + 1, 3)}

    def Kab(a, b):
        return K[(min(a, b), max(a, b))]

    L = []
    for a in range(3):
        s = Kab(a, a) + sum(c[b] * Kab(a, b) for b in range(3) if b != a)
        L.append(n[a] - 0.5 * c[a] * s)
    return p, q, r, L


def t_value(q, r, L, x):
    """T at local coordinates x = (x~, y~, z~) (arrays broadcastable to the cells)."""
    t = q[0] * x[0] ** 2 + q[1] * x[1] ** 2 + q[2] * x[2] ** 2
    t = t + r[(0, 1)] * x[0] * x[1] + r[(1, 2)] * x[1] * x[2] + r[(0, 2)] * x[0] * x[2]
    return t + L[0] * x[0] + L[1] * x[1] + L[2] * x[2]


def log_cosh(x):
    """ln cosh x without overflow: |x| + ln(1 + exp(-2|x|)) - ln 2."""
    ax = np.abs(x)
    return ax + np.log1p(np.exp(-2.0 * ax)) - np.log(2.0)


def line_integral(a, g, d, beta, s0, s1):
    """Integral of (1 + tanh(beta (a s + g + d))) / 2 over s in [s0, s1], exactly (App. A.1.2:
    the one-dimensional antiderivative in log cosh)."""
    return 0.5 * (s1 - s0) + (log_cosh(beta * (a * s1 + g + d)) - log_cosh(beta * (a * s0 + g + d))) / (2.0 * beta * a)


def box_integral(rec, lo, hi, beta):
    """Integral of H over the box prod_a [lo_a, hi_a] of every cell (lo, hi: lists of 3
    arrays or scalars): exact along the cell's p, two-point Gauss along the other two (V4-V6)."""
    p, q, r, L, d = rec["p"], rec["q"], rec["r"], rec["L"], rec["d"]
    out = np.zeros(np.shape(p))
    with np.errstate(divide="ignore", invalid="ignore"):     # cells of another case: masked below
        return _box_integral(p, q, r, L, d, lo, hi, beta, out)


def _box_integral(p, q, r, L, d, lo, hi, beta, out):
    for pp in range(3):
        mask = p == pp
        if not np.any(mask):
            continue
        o1, o2 = [b for b in range(3) if b != pp]
        acc = 0.0
        for t1 in GAUSS:
            for t2 in GAUSS:
                x = [None, None, None]
                x[o1] = lo[o1] + (hi[o1] - lo[o1]) * t1
                x[o2] = lo[o2] + (hi[o2] - lo[o2]) * t2
                x[pp] = 0.0
                g = t_value(q, r, L, x)
                w = 0.25 * (hi[o1] - lo[o1]) * (hi[o2] - lo[o2])
                acc = acc + w * line_integral(L[pp], g, d, beta, lo[pp], hi[pp])
        out = np.where(mask, acc, out)
    return out


def cell_volume_of_h(rec, d, beta):
    """The volume equation's left side (V5): the quadrature of H over the unit cell at d."""
    r2 = dict(rec)
    r2["d"] = d
    z, o = np.zeros(np.shape(d)), np.ones(np.shape(d))
    return box_integral(r2, [z, z, z], [o, o, o], beta)


def reconstruct(phi, beta, eps=EPS_PURE):
    """The MTHINC reconstruction of every cell (App. A.1): uniform mask (V8), case p,
    coefficients of T and d_th (V5, by bisection on the monotone volume equation)."""
    _, n, K = youngs(phi)
    m = youngs_m32(phi)
    zero = (m[0] == 0) & (m[1] == 0) & (m[2] == 0)
    uniform = (phi <= eps) | (phi >= 1.0 - eps) | zero
    # uniform cells never use T; give them a plane normal to x so that no division by a zero
    # slope occurs in the vectorised quadrature
    n = [np.where(uniform, 1.0 if a == 0 else 0.0, n[a]) for a in range(3)]
    m = [np.where(uniform, 1.0 if a == 0 else 0.0, m[a]) for a in range(3)]
    K = {k: np.where(uniform, 0.0, v) for k, v in K.items()}
    p, q, r, L = polynomial(n, K, m)
    rec = {"p": p, "q": q, "r": r, "L": L, "n": n, "m": m, "K": K, "uniform": uniform, "phi": phi}
    # bracket: |T| on the unit cell is at most the sum of the coefficients' magnitudes
    tmax = sum(np.abs(q[a]) + np.abs(L[a]) for a in range(3)) + sum(np.abs(v) for v in r.values())
    lo = -tmax - 40.0 / beta
    hi = tmax + 40.0 / beta
    target = np.where(uniform, 0.5, phi)
    for _ in range(80):                      # bracket width ~1e2 / 2^80: below FP64 rounding
        mid = 0.5 * (lo + hi)
        v = cell_volume_of_h(rec, mid, beta)
        below = v < target
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    rec["d"] = 0.5 * (lo + hi)
    return rec


def quartic_coefficients(rec, beta):
    """The paper's quartic in D = exp(2 beta d_th) (V5): alpha_0 .. alpha_4 per cell."""
    p, q, r, L, phi = rec["p"], rec["q"], rec["r"], rec["L"], rec["phi"]
    A = np.exp(2.0 * beta * np.choose(p, L))
    a = np.choose(p, L)
    Q = np.exp(4.0 * beta * a * (2.0 * phi - 1.0))
    G = []
    for t1 in GAUSS:
        for t2 in GAUSS:
            gq = np.zeros(np.shape(phi))
            for pp in range(3):
                o1, o2 = [b for b in range(3) if b != pp]
                x = [0.0, 0.0, 0.0]
                x[o1], x[o2] = t1, t2
                gq = np.where(p == pp, t_value(q, r, L, x), gq)
            G.append(np.exp(2.0 * beta * gq))
    e = [np.ones(np.shape(phi)), G[0] + G[1] + G[2] + G[3],
         G[0] * G[1] + G[0] * G[2] + G[0] * G[3] + G[1] * G[2] + G[1] * G[3] + G[2] * G[3],
         G[0] * G[1] * G[2] + G[0] * G[1] * G[3] + G[0] * G[2] * G[3] + G[1] * G[2] * G[3],
         G[0] * G[1] * G[2] * G[3]]
    return [e[k] * (A ** k - A * A * Q) for k in range(5)]


# ---------------------------------------------------------- fluxes and split (Sec. 3.1, A.2)

def fluxes(rec, vel, dt, h, a, beta):
    """F at the faces i+1/2 along direction a (stored at cell i): the integral of H of the
    upwind cell over the swept box (V6), as a fraction of the cell volume, signed with u."""
    c = vel * dt / h
    if np.any(np.abs(c) > 1.0):
        raise ValueError("CFL above 1 along a split direction")
    one, zero = np.ones(np.shape(c)), np.zeros(np.shape(c))
    # u >= 0: the lower cell i, box [1 - c, 1] along a
    lo = [zero, zero, zero]
    hi = [one, one, one]
    lo[a] = 1.0 - np.maximum(c, 0.0)
    f_lo = box_integral(rec, lo, hi, beta)
    f_lo = np.where(rec["uniform"], rec["phi"] * np.maximum(c, 0.0), f_lo)
    # u < 0: the upper cell i+1, box [0, -c] along a
    up = {k: (sh(v, 1, a) if isinstance(v, np.ndarray) else v) for k, v in rec.items()
          if k in ("p", "d", "uniform", "phi")}
    up["q"] = [sh(v, 1, a) for v in rec["q"]]
    up["L"] = [sh(v, 1, a) for v in rec["L"]]
    up["r"] = {k: sh(v, 1, a) for k, v in rec["r"].items()}
    lo = [zero, zero, zero]
    hi = [one, one, one]
    hi[a] = np.maximum(-c, 0.0)
    f_up = box_integral(up, lo, hi, beta)
    f_up = np.where(up["uniform"], up["phi"] * np.maximum(-c, 0.0), f_up)
    return np.where(c >= 0.0, f_lo, -f_up)


def split(phi_s, vel, dt, h, a, beta):
    """One directional split (Eq. phi_split): reconstruct phi_s, fluxes along a, and
    phi^a = (phi^s - (F_{i+1/2} - F_{i-1/2})) / (1 - dt/h (u_{i+1/2} - u_{i-1/2}))."""
    rec = reconstruct(phi_s, beta)
    F = fluxes(rec, vel, dt, h, a, beta)
    return (phi_s - (F - sh(F, -1, a))) / (1.0 - dt / h * (vel - sh(vel, -1, a)))


def vof_step(phi, u, v, w, dt, beta, dx, dy, dz):
    """One VoF step (App. A, overall algorithm; Sec. 3.1): splits x, y, z (V9), then the
    divergence correction phi^{n+1} = phi^z - sum_p (dt/dl_p) phi^p (u_+ - u_-)_p
    (Eq. vof_corr_step).  Returns (phi^{n+1}, (phi^x, phi^y, phi^z))."""
    vel, hs = (u, v, w), (dx, dy, dz)
    stages = []
    s = phi
    for a in range(3):
        s = split(s, vel[a], dt, hs[a], a, beta)
        stages.append(s)
    out = stages[2].copy()
    for a in range(3):
        out = out - dt / hs[a] * stages[a] * (vel[a] - sh(vel[a], -1, a))
    return out, tuple(stages)
