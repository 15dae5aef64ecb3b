"""FP64 reference gradient of the time-averaged flux (test infrastructure only).

A second, independent implementation of the DD-TR step of ``lbe_oracle.c``,
written with plain PyTorch CPU tensor operations in float64 so that autograd
gives the exact discrete adjoint of the whole step (shell force, contact
values, collision, streaming).  Its forward pass is checked against the C
oracle; its gradient is checked against central finite differences of the C
oracle.  Only the test suite uses it.

Objective (flux through a plane, averaged over the steps, Sec. "Channel flow
with a bottleneck"):  Phi = (1/T) sum_{t<T} sum_a sum_{plane, fluid} J^a_axis(t),
with J the physical momentum of step t's moments.  Parameters: the per-node
wall-potential amplitude amp(r) (V^a += amp phi for every species) and a body
force g added to every species.
"""
import math

import numpy as np
import torch

from . import lattice, shell, shell_weight, ball

KT = 1.0 / 3.0
CS2 = 1.0 / 3.0


def _site_index(shape, periodic, dx, dy, dz):
    """Index array of node (x+dx, y+dy, z+dz) for every node, -1 outside closed axes."""
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X, Y, Z = x.reshape(-1) + dx, y.reshape(-1) + dy, z.reshape(-1) + dz
    ok = np.ones(X.shape, bool)
    for v, n, per in ((X, nx, periodic[0]), (Y, ny, periodic[1]), (Z, nz, periodic[2])):
        if per:
            v %= n
        else:
            ok &= (v >= 0) & (v < n)
    idx = np.where(ok, X + nx * (Y + ny * Z), -1)
    return idx


class Model:
    """Static tables of one lattice: neighbour indices, shells, balls (all built with numpy)."""

    def __init__(self, shape, periodic, sigmas, taus, solid, phi, V, consistent=False):
        self.shape = tuple(shape)
        self.periodic = tuple(periodic)
        nx, ny, nz = self.shape
        self.N = nx * ny * nz
        self.M = len(sigmas)
        self.sigmas = list(sigmas)
        self.taus = list(taus)
        self.consistent = consistent
        c, w, opp = lattice()
        self.c = torch.tensor(c, dtype=torch.float64)
        self.w = torch.tensor(w, dtype=torch.float64)
        self.ci = c
        self.opp = opp
        self.solid = torch.tensor(np.asarray(solid).reshape(-1) != 0)
        self.fluid = ~self.solid
        self.phi = torch.tensor(np.asarray(phi, dtype=np.float64).reshape(-1))
        self.V = torch.tensor(np.asarray(V, dtype=np.float64).reshape(self.M, -1))
        N = self.N
        sol = np.asarray(solid).reshape(-1) != 0
        # pull streaming with mid-point bounce-back: streamed_p(r) = post_p(r - c_p) or post_opp(p)(r)
        src = np.zeros((19, N), dtype=np.int64)
        for p in range(19):
            j = _site_index(self.shape, self.periodic, -c[p, 0], -c[p, 1], -c[p, 2])
            blocked = (j < 0) | sol[np.maximum(j, 0)]
            src[p] = np.where(blocked, opp[p] * N + np.arange(N), p * N + np.maximum(j, 0))
        self.stream_src = torch.tensor(src)
        # gradient stencil neighbours (clamped to the node itself outside closed axes)
        gidx = np.zeros((19, N), dtype=np.int64)
        for p in range(19):
            j = _site_index(self.shape, self.periodic, c[p, 0], c[p, 1], c[p, 2])
            gidx[p] = np.where(j < 0, np.arange(N), j)
        self.grad_idx = torch.tensor(gidx)
        # balls and shells (index N points at an appended zero)
        self.ball_idx = []
        for b in range(self.M):
            d = ball(0.5 * self.sigmas[b])
            idx = np.stack([_site_index(self.shape, self.periodic, *e) for e in d])
            idx = np.where(idx < 0, N, idx)
            self.ball_idx.append(torch.tensor(idx))
        self.pairs = []
        for a in range(self.M):
            for b in range(self.M):
                sab = 0.5 * (self.sigmas[a] + self.sigmas[b])
                if not sab > 0:
                    continue
                K = shell(sab)
                idx = np.stack([_site_index(self.shape, self.periodic, *e) for e in K])
                idx = np.where(idx < 0, N, idx)
                L = np.sqrt((K.astype(float) ** 2).sum(1))
                ehat = torch.tensor(K / L[:, None], dtype=torch.float64)
                self.pairs.append((a, b, sab, torch.tensor(idx), ehat, shell_weight(sab)))

    # ------------------------------------------------------------------
    def forces(self, amp, gbody):
        """F^a = -grad_h (V^a + amp phi) + g^a, [M, 3, N]."""
        out = []
        for a in range(self.M):
            Vt = self.V[a] + amp * self.phi
            nb = Vt[self.grad_idx]  # [19, N]
            grad = torch.einsum("p,pc,pn->cn", self.w, self.c, nb) / CS2
            out.append(-grad + gbody[a][:, None])
        return torch.stack(out)

    def _ext(self, x):
        return torch.cat([x, x.new_zeros(1)])

    def step(self, f, g, F, axis, plane):
        """One DD-TR step from streamed populations f, g [M, 19, N]; returns (f', g', flux of this step)."""
        M, N = self.M, self.N
        fl = self.fluid.to(torch.float64)
        n = f.sum(1) * fl[None, :]
        # contact values
        xi2 = torch.zeros(N, dtype=torch.float64)
        xi3 = torch.zeros(N, dtype=torch.float64)
        for b in range(M):
            nb = self._ext(n[b] * fl)[self.ball_idx[b]].mean(0)
            s = self.sigmas[b]
            xi2 = xi2 + math.pi / 6 * s * s * nb
            xi3 = xi3 + math.pi / 6 * s ** 3 * nb
        i1 = 1.0 / (1.0 - xi3)
        gp = {}
        for a in range(M):
            for b in range(M):
                sa, sb = self.sigmas[a], self.sigmas[b]
                s = sa * sb / (sa + sb) if sa + sb > 0 else 0.0
                gp[(a, b)] = i1 + 3 * s * xi2 * i1 ** 2 + 2 * s * s * xi2 ** 2 * i1 ** 3
        # shell force
        C = [torch.zeros(3, N, dtype=torch.float64) for _ in range(M)]
        for (a, b, sab, idx, ehat, wab) in self.pairs:
            nbx = self._ext(n[b] * fl)[idx]  # [K, N]
            gab = gp[(a, b)]
            gbar = 0.5 * (gab[None, :] + self._ext(gab)[idx])
            ssum = torch.einsum("kc,kn->cn", ehat, gbar * nbx)
            C[a] = C[a] + (-KT * n[a] * fl * sab * sab * wab)[None, :] * ssum
        C = torch.stack(C)
        # moments
        Pit = g.sum(1)
        Jt = torch.einsum("pc,apn->acn", self.c, g)
        nF = n[:, None, :] * F
        J = Jt + 0.5 * nF if self.consistent else Jt + 0.5 * (C + nF)
        safe = torch.where(n > 0, n, torch.ones_like(n))
        ua = torch.where((n > 0)[:, None, :], J / safe[:, None, :], torch.zeros_like(J))
        Cu = (C * ua).sum(1)
        Pi = Pit + 1.5 * Cu if self.consistent else Pit - 0.5 * Cu
        ntot = n.sum(0)
        u = torch.where((ntot > 0)[None, :], J.sum(0) / torch.where(ntot > 0, ntot, torch.ones_like(ntot))[None, :],
                        torch.zeros_like(J[0]))
        # flux of this step
        coord = self._coord(axis)
        on = (coord == plane) & self.fluid
        flux = (J[:, axis, :] * on.to(torch.float64)[None, :]).sum()
        # collision with the Hermite tensors written out (Sec. "Hard sphere fluid mixture")
        fs, gs = [], []
        H1 = self.c / CS2  # [19, 3]
        eye = torch.eye(3, dtype=torch.float64)
        H2 = (self.c[:, :, None] * self.c[:, None, :] - CS2 * eye[None]) / (2 * CS2 * CS2)  # [19, 3, 3]
        for a in range(M):
            om = 1.0 / (self.taus[a] - 0.5)
            na, Pa, uaa, Ca, nFa = n[a], Pi[a], ua[a], C[a], nF[a]
            t1 = torch.einsum("pc,cn->pn", H1, na[None, :] * uaa)
            T2 = 2 * uaa[:, None, :] * u[None, :, :] - u[:, None, :] * u[None, :, :]  # [3, 3, N]
            t2 = torch.einsum("pcd,cdn->pn", H2, na[None, None, :] * T2)
            feq = self.w[:, None] * (na[None, :] + t1 + t2)
            geq = self.w[:, None] * (Pa[None, :] + t1 + t2)
            H2u = torch.einsum("pcd,dn->pcn", H2, uaa)
            Sf = self.w[:, None] * torch.einsum("cn,pcn->pn", Ca + nFa, H1[:, :, None] + 2 * H2u)
            Sg = self.w[:, None] * (torch.einsum("cn,pcn->pn", Ca, uaa[None] / CS2 + 4 * H2u)
                                    + torch.einsum("cn,pcn->pn", nFa, H1[:, :, None] + 2 * H2u))
            fa = f[a] + (om * (feq - f[a]) + Sf) / (1 + 0.5 * om)
            ga = g[a] + (om * (geq - g[a]) + Sg) / (1 + 0.5 * om)
            fs.append(fa * fl[None, :])
            gs.append(ga * fl[None, :])
        post_f = torch.stack(fs).reshape(M, -1)
        post_g = torch.stack(gs).reshape(M, -1)
        nf = post_f[:, self.stream_src] * fl[None, None, :]
        ng = post_g[:, self.stream_src] * fl[None, None, :]
        return nf, ng, flux

    def _coord(self, axis):
        nx, ny, nz = self.shape
        i = torch.arange(self.N)
        return [i % nx, (i // nx) % ny, i // (nx * ny)][axis]


def flux_objective(model, f0, g0, amp, gshift, gbody, nsteps, axis, plane, ckpt_every=0):
    """Phi = (1/T) sum_t flux_t starting from streamed populations f0, g0 [M, 19, N].
    gshift [3] is added to every species' body force gbody [M][3]."""
    gb = torch.stack([torch.as_tensor(np.asarray(gbody[a], dtype=np.float64)) + gshift for a in range(model.M)])
    F = model.forces(amp, gb)
    f, g = f0, g0
    total = torch.zeros((), dtype=torch.float64)

    def one(f, g):
        return model.step(f, g, F, axis, plane)

    for t in range(nsteps):
        if ckpt_every:
            f, g, fl = torch.utils.checkpoint.checkpoint(one, f, g, use_reentrant=False)
        else:
            f, g, fl = one(f, g)
        total = total + fl
    return total / nsteps, f, g


def reference_gradient(shape, periodic, sigmas, taus, solid, phi, V, gbody, n_init, amp, nsteps, axis, plane,
                       consistent=False, ckpt_every=1):
    """(Phi, dPhi/damp [N], dPhi/dg [3]) by autograd through the FP64 torch step."""
    model = Model(shape, periodic, sigmas, taus, solid, phi, V, consistent)
    M, N = model.M, model.N
    w = model.w
    fl = model.fluid.to(torch.float64)
    f0 = torch.stack([w[:, None] * torch.as_tensor(np.asarray(n_init[a], dtype=np.float64))[None, :] * fl[None, :]
                      for a in range(M)])
    g0 = f0.clone()
    amp_t = torch.tensor(np.asarray(amp, dtype=np.float64).reshape(-1), requires_grad=True)
    gs = torch.zeros(3, dtype=torch.float64, requires_grad=True)
    Phi, _, _ = flux_objective(model, f0, g0, amp_t, gs, gbody, nsteps, axis, plane, ckpt_every)
    Phi.backward()
    return float(Phi.detach()), amp_t.grad.numpy().copy(), gs.grad.numpy().copy()


def forward_only(shape, periodic, sigmas, taus, solid, phi, V, gbody, n_init, amp, nsteps, axis, plane,
                 consistent=False):
    model = Model(shape, periodic, sigmas, taus, solid, phi, V, consistent)
    w = model.w
    fl = model.fluid.to(torch.float64)
    f0 = torch.stack([w[:, None] * torch.as_tensor(np.asarray(n_init[a], dtype=np.float64))[None, :] * fl[None, :]
                      for a in range(model.M)])
    with torch.no_grad():
        Phi, f, g = flux_objective(model, f0, f0.clone(), torch.as_tensor(np.asarray(amp, dtype=np.float64)),
                                   torch.zeros(3, dtype=torch.float64), gbody, nsteps, axis, plane)
    return float(Phi), f.numpy(), g.numpy()
