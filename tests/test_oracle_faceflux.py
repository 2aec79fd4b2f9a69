"""The oracle's single-face Riemann flux (used to check sampled faces of
grids too large for the oracle to sweep) is the same function as its full
sweep: on a small torus every interior face of every direction agrees with
the sweep's flux exactly, for the components flux-CT leaves alone."""
import numpy as np

import oracle as O

NOT_B = [0, 1, 2, 3, 4, 8]


def test_face_flux_at_matches_the_sweep():
    og = O.Grid(O.default_params(n1=12, n2=10, n3=6))
    og.init_torus(pert_amp=0.04, seed=3)
    P = og.get_state()[0]
    F, _ = og.fluxes()
    n1, n2, n3 = og.shape
    checked = 0
    for d in range(3):
        for i in range(2, n1 - 1):
            for j in range(2, n2 - 1):
                for k in range(2, n3 - 1):
                    idx = [i, j, k]
                    st = []
                    for o in (-2, -1, 0, 1):
                        z = list(idx)
                        z[d] += o
                        st.append(P[:, z[0], z[1], z[2]])
                    Fo, cw = og.face_flux_at(d, i, j, np.array(st))
                    assert cw >= 0.0
                    assert np.array_equal(Fo[NOT_B], F[d][NOT_B, i, j, k])
                    checked += 1
    assert checked > 500
