"""Oracle of the learned interface correction (not in the paper).

At the deepest Schur level l* = nlev - 2, after the GeMSLR solve has produced
y2 = M_S^{-1} z2 (C_l*^{-1} applied to z2 plus the low-rank term, Alg. 2), a
small 3-D convolutional network N refines it:

    rho = z2 - S_hat y2,   S_hat = C_l* - E_l* (U^{-1} L^{-1}) F_l*   (Sec. 2.4)
    y2 <- y2 + N(rho)

N is trained so that N(rho) ~ S_hat^{-1} rho.  FGMRES tolerates the
resulting variable preconditioner (Sec. 5 set-up: flexible GMRES is used
because the preconditioner may change between iterations).

Network (plain FP64 here): sites = the unknowns of level l*'s tail with
their grid coordinates; every layer is a 27-tap (3x3x3) convolution over the
sites that exist (missing neighbours contribute nothing), with bias; ReLU
after layers 1..3; channels 1 -> C -> C -> C -> 1.  Input and output are
scaled:  N(rho) = (||rho|| / d) * net(rho / ||rho||), with d the mean |diagonal|
of S_hat, so the network works on O(1) values and N is positively homogeneous.

Tap order: t = (dz+1)*9 + (dy+1)*3 + (dx+1).
"""
import numpy as np
import scipy.linalg as sla


def site_neighbors(coords):
    """nbr[s, t] = index of the site at offset t of site s, or -1."""
    coords = np.asarray(coords, dtype=np.int64)
    key = {tuple(c): i for i, c in enumerate(coords)}
    S = len(coords)
    nbr = np.full((S, 27), -1, dtype=np.int64)
    for s, c in enumerate(coords):
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    t = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
                    nbr[s, t] = key.get((c[0] + dx, c[1] + dy, c[2] + dz), -1)
    return nbr


def conv_forward(x, W, b, nbr):
    """y[n, s, co] = b[co] + sum_t sum_ci W[t, ci, co] x[n, nbr[s, t], ci].  x: (N, S, Cin)."""
    N, S, Cin = x.shape
    Cout = W.shape[2]
    y = np.broadcast_to(b, (N, S, Cout)).copy()
    for t in range(27):
        src = nbr[:, t]
        ok = src >= 0
        xs = np.zeros((N, S, Cin))
        xs[:, ok, :] = x[:, src[ok], :]
        y += xs @ W[t]
    return y


def conv_backward(x, W, nbr, dy):
    """Gradients of sum(dy * conv_forward(x, W, b)) with respect to x, W, b."""
    N, S, Cin = x.shape
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for t in range(27):
        src = nbr[:, t]
        ok = src >= 0
        xs = np.zeros((N, S, Cin))
        xs[:, ok, :] = x[:, src[ok], :]
        dW[t] = np.einsum("nsi,nso->io", xs, dy)
        g = dy @ W[t].T                               # (N, S, Cin) at the output site
        np.add.at(dx, (slice(None), src[ok], slice(None)), g[:, ok, :])
    db = dy.sum(axis=(0, 1))
    return dx, dW, db


def init_params(channels=32, seed=0):
    """He-style initialisation from a seeded stream (weights W[l]: (27, Cin, Cout))."""
    import gemslr_inputs
    dims = [1, channels, channels, channels, 1]
    params = []
    for l in range(4):
        cin, cout = dims[l], dims[l + 1]
        n = 27 * cin * cout
        u = gemslr_inputs.uniform01(seed * 100 + l, n)
        bound = np.sqrt(6.0 / (27 * cin)) * (1.0 if l < 3 else 0.1)
        W = ((2.0 * u - 1.0) * bound).reshape(27, cin, cout)
        params.append([W, np.zeros(cout)])
    return params


def net_forward(params, x, nbr):
    """x: (N, S) -> (N, S); returns output and the activations for backward."""
    acts = [x[:, :, None]]
    h = acts[0]
    for l, (W, b) in enumerate(params):
        z = conv_forward(h, W, b, nbr)
        h = np.maximum(z, 0.0) if l < 3 else z
        acts.append(z)
        if l < 3:
            acts.append(h)
    return h[:, :, 0], acts


def net_backward(params, acts, nbr, dout):
    """Gradients of sum(dout * net(x)) for every (W, b)."""
    grads = [None] * 4
    g = dout[:, :, None]
    # acts = [x, z1, h1, z2, h2, z3, h3, z4]
    inputs = [acts[0], acts[2], acts[4], acts[6]]
    pre = [acts[1], acts[3], acts[5], acts[7]]
    for l in range(3, -1, -1):
        if l < 3:
            g = g * (pre[l] > 0.0)
        dx, dW, db = conv_backward(inputs[l], params[l][0], nbr, g)
        grads[l] = (dW, db)
        g = dx
    return grads


def loss_and_grads(params, rho, target, nbr):
    """Mean over samples of ||net(rho) - target||^2 / ||target||^2 (inputs already scaled)."""
    out, acts = net_forward(params, rho, nbr)
    diff = out - target
    den = np.sum(target * target, axis=1)
    loss = float(np.mean(np.sum(diff * diff, axis=1) / den))
    dout = 2.0 * diff / den[:, None] / rho.shape[0]
    return loss, net_backward(params, acts, nbr, dout)


def schur_dense(M, l):
    """S_hat_l = C_l - E_l (L U)^{-1} F_l formed exactly (dense) from the oracle hierarchy."""
    from .ilu import lu_solve
    lv = M.levels[l]
    e = lv["e"]
    C = M.Ahat[e:, e:].toarray()
    F = lv["F"].toarray()
    X = np.column_stack([lu_solve(lv["L"], lv["U"], F[:, j]) for j in range(F.shape[1])])
    return C - lv["E"].toarray() @ X


def interface_stage(M, net, d=None):
    """The in-apply correction of level l* = nlev - 2 as a callable for
    ``OracleGemslr.stage``:

        rho = z2 - S_hat y2,   y2' = y2 + (||rho|| / d) * net(rho / ||rho||)

    with S_hat y2 = C y2 - E (U^{-1} L^{-1}) F y2 (``OracleGemslr.s_hat``, Sec. 2.4)
    and d the mean |diagonal| of S_hat (formed densely when not given).  ``net``
    maps a vector of the level's S sites to S values; ``cnn(params, nbr)``
    gives the network.  rho = 0 leaves y2 unchanged."""
    l = M.nlev - 2
    if d is None:
        d = float(np.mean(np.abs(np.diag(schur_dense(M, l)))))

    def stage(z2, y2):
        rho = z2 - M.s_hat(y2, l)
        nr = float(np.linalg.norm(rho))
        if nr == 0.0:
            return y2
        return y2 + (nr / d) * net(rho / nr)

    return stage


def cnn(params, nbr):
    """The 4-layer network as a map of one site vector (S,) -> (S,)."""
    def f(x):
        out, _ = net_forward(params, np.asarray(x, dtype=np.float64)[None, :], nbr)
        return out[0]
    return f


def level_preconditioner_dense(M, l):
    """M_S^{-1} of level l (C_l^{-1} approximated by the levels below, plus the low-rank term) as a dense matrix."""
    lv = M.levels[l]
    s = M.n - lv["e"]
    I = np.eye(s)
    W, H = lv["W"], lv["H"]
    cols = []
    for j in range(s):
        z = I[:, j]
        u = W @ (H @ (W.T @ z)) if W.shape[1] else 0.0
        cols.append(M.solve_level(z + u, l + 1))
    return np.column_stack(cols)


def training_pairs(M, l, count, seed):
    """(rho, S_hat^{-1} rho) for z2 ~ U[-1,1): rho = z2 - S_hat M_S^{-1} z2."""
    import gemslr_inputs
    S = schur_dense(M, l)
    P = level_preconditioner_dense(M, l)
    s = S.shape[0]
    Z = (2.0 * gemslr_inputs.uniform01(seed, s * count) - 1.0).reshape(count, s)
    R = Z - (S @ (P @ Z.T)).T
    lu = sla.lu_factor(S)
    T = sla.lu_solve(lu, R.T).T
    return R, T, S
