"""Exact rational one-step trace of the two-component Shan-Chen model on a tiny
D2Q9 lattice (ExactSC) and a tiny D3Q19 lattice (ExactSC3), written independently of the oracle (brute force in
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


# --- D3Q19 -------------------------------------------------------------------
# Textbook D3Q19 order: rest, the six axis directions, then the twelve face
# diagonals (xy, xz, yz planes).  Weights 1/3, 1/18, 1/36.
C3 = ([(0, 0, 0)]
      + [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
      + [(a, b, 0) for a in (1, -1) for b in (1, -1)]
      + [(a, 0, b) for a in (1, -1) for b in (1, -1)]
      + [(0, a, b) for a in (1, -1) for b in (1, -1)])
W3 = [Fr(1, 3)] + [Fr(1, 18)] * 6 + [Fr(1, 36)] * 12


def _hermite(c_set, w_set, rho, u):
    """w_i rho [1 + c.u/cs2 + (c_a c_b - cs2 delta_ab) u_a u_b / (2 cs2^2)] in any dimension."""
    d = len(u)
    out = []
    for c, w in zip(c_set, w_set):
        cu = sum(c[a] * u[a] for a in range(d))
        q = sum((c[a] * c[b] - (CS2 if a == b else 0)) * u[a] * u[b] for a in range(d) for b in range(d))
        out.append(w * rho * (1 + cu / CS2 + q / (2 * CS2 * CS2)))
    return out


def _source(c_set, w_set, u, F):
    """Guo's source in Hermite form, w_i [c.F/cs2 + (c_a c_b - cs2 delta_ab)(u_a F_b + F_a u_b)/(2 cs2^2)]."""
    d = len(u)
    out = []
    for c, w in zip(c_set, w_set):
        cF = sum(c[a] * F[a] for a in range(d))
        q = sum((c[a] * c[b] - (CS2 if a == b else 0)) * (u[a] * F[b] + F[a] * u[b])
                for a in range(d) for b in range(d))
        out.append(w * (cF / CS2 + q / (2 * CS2 * CS2)))
    return out


class ExactSC3:
    """The same model on a periodic D3Q19 box, node coordinates (x, y, z);
    f[s][(x, y, z)] is a list of 19 Fractions.  Body force of Eq. kolmo along x
    with the sine of 2 pi y / ny exact for ny in {1, 2, 4}."""

    def __init__(self, nx, ny, nz, tau_A, tau_B, G, body_A=0, guo=False):
        self.n = (nx, ny, nz)
        self.tau = (Fr(tau_A), Fr(tau_B))
        self.G = Fr(G)
        self.A = Fr(body_A)
        self.guo = guo
        quarter = [Fr(0), Fr(1), Fr(0), Fr(-1)]
        assert ny in (1, 2, 4) or self.A == 0
        self.sin_y = [quarter[(4 // ny) * y % 4] if ny in (1, 2, 4) else Fr(0) for y in range(ny)]
        self.nodes = [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)]
        self.f = None

    def _wrap(self, p):
        return tuple(p[a] % self.n[a] for a in range(3))

    def init(self, rhoA, rhoB):
        """Rest equilibrium from rational densities rho[z][y][x]."""
        zero = (Fr(0),) * 3
        self.f = [{(x, y, z): _hermite(C3, W3, Fr(r[z][y][x]), zero) for (x, y, z) in self.nodes}
                  for r in (rhoA, rhoB)]
        return self

    def _moments(self):
        rho = [{p: sum(self.f[s][p]) for p in self.nodes} for s in (0, 1)]
        j = [{p: tuple(sum(fi * c[a] for fi, c in zip(self.f[s][p], C3)) for a in range(3)) for p in self.nodes}
             for s in (0, 1)]
        F = [{}, {}]
        for s in (0, 1):
            o = 1 - s
            for p in self.nodes:
                acc = [Fr(0)] * 3
                for c, w in zip(C3, W3):
                    r = rho[o][self._wrap((p[0] + c[0], p[1] + c[1], p[2] + c[2]))]
                    for a in range(3):
                        acc[a] += w * r * c[a]
                body = (rho[s][p] * self.A * self.sin_y[p[1]], Fr(0), Fr(0))
                F[s][p] = tuple(-self.G * rho[s][p] * acc[a] + body[a] for a in range(3))
        return rho, j, F

    def step(self):
        rho, j, F = self._moments()
        post = [{}, {}]
        for p in self.nodes:
            den = sum(rho[s][p] / self.tau[s] for s in (0, 1))
            if self.guo:
                uc = tuple(sum((j[s][p][a] + F[s][p][a] / 2) / self.tau[s] for s in (0, 1)) / den for a in range(3))
            else:
                uc = tuple(sum(j[s][p][a] / self.tau[s] for s in (0, 1)) / den for a in range(3))
            for s in (0, 1):
                t = self.tau[s]
                if self.guo:
                    fe = _hermite(C3, W3, rho[s][p], uc)
                    src = _source(C3, W3, uc, F[s][p])
                    post[s][p] = [fi - (fi - e) / t + (1 - 1 / (2 * t)) * si
                                  for fi, e, si in zip(self.f[s][p], fe, src)]
                else:
                    ueq = tuple(uc[a] + t * F[s][p][a] / rho[s][p] for a in range(3))
                    fe = _hermite(C3, W3, rho[s][p], ueq)
                    post[s][p] = [fi - (fi - e) / t for fi, e in zip(self.f[s][p], fe)]
        # pull: f_i(x, t+1) = f*_i(x - c_i, t)
        self.f = [{p: [post[s][self._wrap((p[0] - c[0], p[1] - c[1], p[2] - c[2]))][i] for i, c in enumerate(C3)]
                   for p in self.nodes} for s in (0, 1)]
        return self

    def fields(self):
        """rho_A, rho_B, u_phys (three components), p, each a list in z, y, x order (x fastest)."""
        rho, j, F = self._moments()
        out = [[] for _ in range(6)]
        for p in self.nodes:
            a, b = rho[0][p], rho[1][p]
            tot = a + b
            m = [j[0][p][k] + j[1][p][k] + (F[0][p][k] + F[1][p][k]) / 2 for k in range(3)]
            for lst, v in zip(out, (a, b, m[0] / tot, m[1] / tot, m[2] / tot, CS2 * tot + CS2 * self.G * a * b)):
                lst.append(v)
        return out
