"""Exact rational one-step trace of the two-component Shan-Chen model on a tiny
D2Q9 lattice, written independently of the oracle (brute force in
``fractions.Fraction``, pull streaming, textbook velocity order, Hermite form
of the equilibrium).  Used only to pin the oracle.

The model (Sec. 2.1): moments rho_s = sum_i f_is, u' = sum_s j_s/tau_s /
sum_s rho_s/tau_s; force F_s(x) = -G rho_s(x) sum_i w_i rho_s'(x+c_i) c_i
(Eq. FORCE); BGK relaxation to f^eq(rho_s, u' + tau_s F_s/rho_s) (Eq. eq:be)
followed by streaming along c_i on a periodic box.  Optional Kolmogorov body
force (Eq. kolmo, Sec. 4.2): F_s,x += rho_s A sin(2 pi y / ny), kept exact by
allowing only ny in {1, 2, 4}, where the sine takes the values 0 and +-1.
Optional Guo forcing (guo=True), the discrete-forcing cure Sec. 2.3 names:
relaxation to f^eq(rho_s, u_G), u_G = sum_s (j_s + F_s/2)/tau_s / sum_s
rho_s/tau_s, plus (1 - 1/(2 tau_s)) times the source written here in its
Hermite form w_i [c.F/cs2 + (c_a c_b - cs2 delta_ab)(u_a F_b + F_a u_b)/(2 cs2^2)].
"""
from fractions import Fraction as Fr

# Textbook D2Q9 order: rest, E, N, W, S, NE, NW, SW, SE.
C = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
W = [Fr(4, 9)] + [Fr(1, 9)] * 4 + [Fr(1, 36)] * 4
CS2 = Fr(1, 3)


def feq_hermite(rho, u):
    """w_i rho [1 + c.u/cs2 + (c_a c_b - cs2 delta_ab) u_a u_b / (2 cs2^2)]."""
    out = []
    for (cx, cy), w in zip(C, W):
        cu = cx * u[0] + cy * u[1]
        q = (cx * cx - CS2) * u[0] * u[0] + 2 * cx * cy * u[0] * u[1] + (cy * cy - CS2) * u[1] * u[1]
        out.append(w * rho * (1 + cu / CS2 + q / (2 * CS2 * CS2)))
    return out


class ExactSC:
    """f[s][y][x] is a list of 9 Fractions."""

    def __init__(self, nx, ny, tau_A, tau_B, G, body_A=0, guo=False):
        self.guo = guo
        self.nx, self.ny = nx, ny
        self.tau = (Fr(tau_A), Fr(tau_B))
        self.G = Fr(G)
        self.A = Fr(body_A)
        # sin(2 pi y / ny) for ny = 4: 0, 1, 0, -1; ny = 1, 2: zeros
        quarter = [Fr(0), Fr(1), Fr(0), Fr(-1)]
        assert ny in (1, 2, 4) or self.A == 0
        self.sin_y = [quarter[(4 // ny) * y % 4] if ny in (1, 2, 4) else Fr(0) for y in range(ny)]
        self.f = None

    def init(self, rhoA, rhoB):
        """Rest equilibrium from rational density grids rho[y][x]."""
        zero = (Fr(0), Fr(0))
        self.f = [[[feq_hermite(Fr(r[y][x]), zero) for x in range(self.nx)] for y in range(self.ny)]
                  for r in (rhoA, rhoB)]
        return self

    def _moments(self):
        rho = [[[sum(self.f[s][y][x]) for x in range(self.nx)] for y in range(self.ny)] for s in (0, 1)]
        j = [[[(sum(fi * c[0] for fi, c in zip(self.f[s][y][x], C)),
                sum(fi * c[1] for fi, c in zip(self.f[s][y][x], C)))
               for x in range(self.nx)] for y in range(self.ny)] for s in (0, 1)]
        F = [[[None] * self.nx for _ in range(self.ny)] for _ in (0, 1)]
        for s in (0, 1):
            o = 1 - s
            for y in range(self.ny):
                for x in range(self.nx):
                    sx = sy = Fr(0)
                    for (cx, cy), w in zip(C, W):
                        r = rho[o][(y + cy) % self.ny][(x + cx) % self.nx]
                        sx += w * r * cx
                        sy += w * r * cy
                    F[s][y][x] = (-self.G * rho[s][y][x] * sx + rho[s][y][x] * self.A * self.sin_y[y],
                                  -self.G * rho[s][y][x] * sy)
        return rho, j, F

    @staticmethod
    def source_hermite(u, F):
        out = []
        for (cx, cy), w in zip(C, W):
            cF = cx * F[0] + cy * F[1]
            q = ((cx * cx - CS2) * 2 * u[0] * F[0] + cx * cy * (u[0] * F[1] + F[0] * u[1])
                 + cy * cx * (u[1] * F[0] + F[1] * u[0]) + (cy * cy - CS2) * 2 * u[1] * F[1])
            out.append(w * (cF / CS2 + q / (2 * CS2 * CS2)))
        return out

    def _step_guo(self, rho, j, F):
        post = [[[None] * self.nx for _ in range(self.ny)] for _ in (0, 1)]
        for y in range(self.ny):
            for x in range(self.nx):
                den = sum(rho[s][y][x] / self.tau[s] for s in (0, 1))
                uG = tuple(sum((j[s][y][x][a] + F[s][y][x][a] / 2) / self.tau[s] for s in (0, 1)) / den
                           for a in (0, 1))
                for s in (0, 1):
                    fe = feq_hermite(rho[s][y][x], uG)
                    src = self.source_hermite(uG, F[s][y][x])
                    t = self.tau[s]
                    post[s][y][x] = [fi - (fi - e) / t + (1 - 1 / (2 * t)) * si
                                     for fi, e, si in zip(self.f[s][y][x], fe, src)]
        return post

    def step(self):
        rho, j, F = self._moments()
        if self.guo:
            post = self._step_guo(rho, j, F)
            self.f = [[[[post[s][(y - cy) % self.ny][(x - cx) % self.nx][i] for i, (cx, cy) in enumerate(C)]
                        for x in range(self.nx)] for y in range(self.ny)] for s in (0, 1)]
            return self
        post = [[[None] * self.nx for _ in range(self.ny)] for _ in (0, 1)]
        for y in range(self.ny):
            for x in range(self.nx):
                den = sum(rho[s][y][x] / self.tau[s] for s in (0, 1))
                up = tuple(sum(j[s][y][x][a] / self.tau[s] for s in (0, 1)) / den for a in (0, 1))
                for s in (0, 1):
                    r = rho[s][y][x]
                    ueq = tuple(up[a] + self.tau[s] * F[s][y][x][a] / r for a in (0, 1))
                    fe = feq_hermite(r, ueq)
                    post[s][y][x] = [fi - (fi - e) / self.tau[s] for fi, e in zip(self.f[s][y][x], fe)]
        # pull: f_i(x, t+1) = f*_i(x - c_i, t)
        self.f = [[[[post[s][(y - cy) % self.ny][(x - cx) % self.nx][i] for i, (cx, cy) in enumerate(C)]
                    for x in range(self.nx)] for y in range(self.ny)] for s in (0, 1)]
        return self

    def fields(self):
        """rho_A, rho_B, u_phys = (sum j + sum F / 2) / rho, p = cs2 rho + cs2 G rho_A rho_B."""
        rho, j, F = self._moments()
        rA, rB, ux, uy, p = [], [], [], [], []
        for y in range(self.ny):
            for x in range(self.nx):
                a, b = rho[0][y][x], rho[1][y][x]
                tot = a + b
                m = [j[0][y][x][k] + j[1][y][x][k] + (F[0][y][x][k] + F[1][y][x][k]) / 2 for k in (0, 1)]
                rA.append(a)
                rB.append(b)
                ux.append(m[0] / tot)
                uy.append(m[1] / tot)
                p.append(CS2 * tot + CS2 * self.G * a * b)
        return rA, rB, ux, uy, p
