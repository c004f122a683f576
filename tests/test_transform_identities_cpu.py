"""The transform-domain identities the field paths are built on, checked on the CPU in
FP64 against the oracle's direct sum h_n = sum_m W~(n - m) s_m (Sec. 2.1, Eq. 2) at the
update sites of one sub-step (Sec. 3.1: the sites o + l D of cell offset o).  These are
the derivations the kernels rest on, written out with numpy from their definitions:

  * sub-lattice spectra (the spectral path, any C = L/l): with C x C DFTs S_e(K) of the
    spin sub-lattices and T_d(K) of the W~ sub-lattices, the field at the sites of offset o
    is the inverse DFT of H_o(K) = sum_e w^(K.sigma) T_((o - e) mod l)(K) S_e(K), sigma
    marking where o - e wraps into [0, l);
  * the 2 x 2 cell grid at L = 2l (the tensor path's spectral operands and the direct
    kernel's transform-domain sums) is that identity with w = -1;
  * the field change at the cells of offset o from moves at the cells of offset e
    (the sub-step kernel's pushes) is (1/4) sum_k (-1)^(k.D) U_(o-e)(k) S^_e(k), with
    U_d(k) = sum_P (-1)^(k.P) W~(d + l P), and W~(d + l P) is the inverse 2 x 2 transform
    of U_d (its pair-energy table);
  * W~ is even, so its 2D transform is real (the FFT path), and the field at the rows
    y_i = o_y + l i needs only the transform's rows summed by k_y mod C (the cluster path);
  * a window's field is the stale field at its start plus the change from the moves it
    accepted in earlier sub-steps (every windowed path).
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1211_6234_b300 import inputs


def apply_w(w, v):
    """W~ (xx, xy, yy, zz) applied to a spin vector v (components first)."""
    return np.stack([w[0] * v[0] + w[1] * v[1], w[1] * v[0] + w[2] * v[1], w[3] * v[2]])


def wt(W, x, y):
    """W~ at displacement (x, y), periodic in L: [4]."""
    L = W.shape[-1]
    return W[:, y % L, x % L]


@pytest.mark.parametrize("L,l", [(8, 4), (12, 4), (12, 3), (16, 4), (12, 6)])
def test_sub_lattice_spectra_give_the_field_at_a_sub_steps_sites(L, l):
    C = L // l
    W = orc.wtilde(L, 8, True)
    s = inputs.random_spins(L, 1, seed=L + l)[0]
    h = orc.field(W, s)
    w = np.exp(-2j * np.pi / C)
    K = np.arange(C)
    F = w ** np.outer(K, K)                                       # F[K, D] = w^(K D)

    def dft2(f):                                                  # f[..., Dy, Dx] -> [..., Ky, Kx]
        return np.einsum("yb,...ba,xa->...yx", F, f, F)

    # S_e(K) for every cell offset e = (ex, ey), T_d(K) for every d in [0, l)^2
    S = {(ex, ey): dft2(s[:, ey::l, ex::l]) for ey in range(l) for ex in range(l)}
    T = {}
    for dy in range(l):
        for dx in range(l):
            g = np.array([[wt(W, dx + l * Dx, dy + l * Dy) for Dx in range(C)] for Dy in range(C)])
            T[(dx, dy)] = dft2(np.moveaxis(g, -1, 0))             # [4][Ky][Kx]
    rng = np.random.default_rng(L * l)
    for ox, oy in [(0, 0), (l - 1, l - 1)] + [tuple(rng.integers(0, l, 2)) for _ in range(3)]:
        H = np.zeros((3, C, C), complex)
        for (ex, ey), Se in S.items():
            sx, sy = int(ox < ex), int(oy < ey)
            phase = w ** (np.add.outer(K * sy, K * sx))           # w^(K . sigma)
            H += phase * apply_w(T[((ox - ex) % l, (oy - ey) % l)], Se)
        Finv = np.conj(F) / C
        hq = np.einsum("yb,cba,xa->cyx", Finv, H, Finv).real      # field at o + l (Dx, Dy)
        np.testing.assert_allclose(hq, h[:, oy::l, ox::l], rtol=0, atol=1e-12 * np.abs(h).max())


@pytest.mark.parametrize("L", [8, 12, 16])
def test_cell_grid_pushes_and_pair_energies_at_L_equal_2l(L):
    l = L // 2
    W = orc.wtilde(L, 8, True)
    s = inputs.random_spins(L, 1, seed=3 * L)[0]
    rng = np.random.default_rng(L)
    had = np.array([[1, 1, 1, 1], [1, -1, 1, -1], [1, 1, -1, -1], [1, -1, -1, 1]], float)  # (-1)^(k.D)
    for _ in range(6):
        ex, ey, ox, oy = (int(v) for v in rng.integers(0, l, 4))
        delta = np.zeros_like(s)
        for D in range(4):                                        # moves at the four cells of e
            x, y = ex + l * (D & 1), ey + l * (D >> 1)
            v = rng.normal(size=3)
            delta[:, y, x] = v / np.linalg.norm(v) - s[:, y, x]
        dh = orc.field(W, s + delta) - orc.field(W, s)
        d = (ox - ex, oy - ey)                                    # in (-l, l)^2, not wrapped
        Wp = np.array([wt(W, d[0] + l * (P & 1), d[1] + l * (P >> 1)) for P in range(4)])   # [P][4]
        U = had @ Wp                                              # U_d(k) = sum_P (-1)^(k.P) W~(d + l P)
        np.testing.assert_allclose(had @ U / 4, Wp, rtol=0, atol=1e-14)   # the pair table's inverse
        Shat = np.array([sum(had[k, D] * delta[:, ey + l * (D >> 1), ex + l * (D & 1)] for D in range(4))
                         for k in range(4)])                      # [k][3]
        for D in range(4):
            pred = sum(had[k, D] * apply_w(U[k], Shat[k]) for k in range(4)) / 4
            got = dh[:, oy + l * (D >> 1), ox + l * (D & 1)]
            np.testing.assert_allclose(pred, got, rtol=0, atol=1e-12 * np.abs(dh).max())


@pytest.mark.parametrize("L,l", [(16, 4), (16, 8), (32, 8)])
def test_real_transform_of_w_and_rows_grouped_by_ky_mod_C(L, l):
    C = L // l
    W = orc.wtilde(L, 8, True)
    s = inputs.random_spins(L, 1, seed=L + 5)[0]
    h = orc.field(W, s)
    What = np.fft.fft2(W)                                         # [4][ky][kx]
    assert np.abs(What.imag).max() < 1e-10 * np.abs(What.real).max()    # W~ is even
    Sh = np.fft.fft2(s)
    Hh = np.stack([What[0] * Sh[0] + What[1] * Sh[1], What[1] * Sh[0] + What[2] * Sh[1], What[3] * Sh[2]])
    np.testing.assert_allclose(np.fft.ifft2(Hh).real, h, rtol=0, atol=1e-11 * np.abs(h).max())
    ky = np.arange(L)
    for ox, oy in [(1, 2), (l - 1, 0)]:
        # P(kx, r) = sum over ky = r (mod C) of e^(2 pi i ky oy / L) H^(kx, ky); then the rows
        # y_i = oy + l i need only the C-point transform over r
        ph = np.exp(2j * np.pi * ky * oy / L)
        P = np.stack([(ph[ky % C == r, None] * Hh[:, ky % C == r, :]).sum(axis=1) for r in range(C)], axis=1)
        i = np.arange(C)
        G = np.einsum("ir,crx->cix", np.exp(2j * np.pi * np.outer(i, np.arange(C)) / C), P)
        kx = np.arange(L)
        xs = ox + l * np.arange(C)
        hq = np.einsum("jx,cix->cij", np.exp(2j * np.pi * np.outer(xs, kx) / L), G).real / (L * L)
        np.testing.assert_allclose(hq, h[:, oy::l, ox::l], rtol=0, atol=1e-11 * np.abs(h).max())


@pytest.mark.parametrize("L,l,B,schedule", [(16, 8, 16, 0), (16, 4, 8, 0), (12, 6, 12, 0), (16, 8, 16, 1)])
def test_window_field_is_the_stale_field_plus_the_windows_earlier_moves(L, l, B, schedule):
    """The windowed paths evaluate the field at all of a window's sites once, on the state
    at the window's start, and add per sub-step the change from the moves the window
    accepted in earlier sub-steps (linearity of Eq. 2; a sub-step's own sites are decided
    together from the pre-step state, Sec. 3.1).  Along the oracle's own sweep, whose every
    sub-step takes the full field of the current state, that decomposition reproduces the
    field of every attempt, also under the with-replacement schedule where a site may recur."""
    n = (L // l) ** 2
    p = orc.params(L, l, 1.0, 0.1, 0.8, 0.0, 0.6, proposal=0, cone=0.5, schedule=schedule, seed=9)
    W = orc.wtilde(L, 8, True)
    s0 = inputs.random_spins(L, 1, seed=4)[0]
    o = orc.sweeps(p, W, s0, 0, 1, trace=True)
    cur = s0.reshape(3, -1).copy()
    scale = np.abs(o["h"]).max()
    for w0 in range(0, l * l, B):
        h0 = orc.field(W, cur.reshape(3, L, L)).reshape(3, -1)
        moves = []                                                # (x, y, change) accepted in the window
        for k in range(w0, w0 + B):
            rows = range(k * n, (k + 1) * n)
            for a in rows:
                q = int(o["q"][a])
                qx, qy = q % L, q // L
                pred = h0[:, q].copy()
                for px, py, dv in moves:
                    pred += apply_w(wt(W, qx - px, qy - py), dv)
                np.testing.assert_allclose(pred, o["h"][a], rtol=0, atol=1e-12 * scale)
            for a in rows:                                        # then the sub-step's accepted moves
                if o["acc"][a]:
                    q = int(o["q"][a])
                    moves.append((q % L, q // L, o["S"][a] - cur[:, q]))
                    cur[:, q] = o["S"][a]
    np.testing.assert_array_equal(cur.reshape(3, L, L), o["s"])
