"""The seeded input generators (no arithmetic of the method): the AMA source
translations keep the SAP decomposition (Sec. 2.2, end: each of the domains
Omega and Omega* must map onto itself), and the fields have the stated
structure."""
import numpy as np
import pytest

from paper_1605_00564_gb300 import synth


@pytest.mark.parametrize("dims,block,n_g", [((64, 32, 32, 32), (4, 4, 4, 4), 8), ((48, 24, 24, 24), (4, 4, 4, 4), 8),
                                            ((16, 8, 8, 8), (4, 4, 4, 4), 2), ((96, 48, 48, 48), (6, 6, 6, 6), 8)])
def test_ama_shifts_preserve_the_domains(dims, block, n_g):
    shifts = synth.ama_source_shifts(dims, n_g, block)
    assert len(shifts) == n_g and len(set(shifts)) == n_g           # distinct positions
    assert shifts[0] == (0, 0, 0, 0)                                 # N_org = 1 at the origin
    for g in shifts:
        nblk = 0
        for mu in range(4):
            assert 0 <= g[mu] < dims[mu]
            assert g[mu] % block[mu] == 0                            # blocks map onto blocks
            nblk += g[mu] // block[mu]
        assert nblk % 2 == 0                                         # Omega -> Omega, not Omega*


def test_gauge_field_is_special_unitary_and_seeded():
    dims = (4, 4, 4, 6)
    U = synth.gauge_field(dims, 0.3, 11)
    assert U.shape == tuple(synth.lattice_shape(dims)) + (4, 3, 3)    # (T, Z, Y, X, mu, row, col)
    eye = np.eye(3)
    uu = np.einsum("...ji,...jk->...ik", U.conj(), U)
    assert np.abs(uu - eye).max() < 1e-12
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-12
    assert np.array_equal(U, synth.gauge_field(dims, 0.3, 11))
    assert not np.array_equal(U, synth.gauge_field(dims, 0.3, 12))


def test_point_sources_are_the_12_unit_vectors():
    dims = (4, 4, 4, 4)
    src = (1, 2, 3, 0)
    eta = synth.point_sources(dims, src)
    assert eta.shape == (12,) + dims[:1] + dims[:0:-1] + (4, 3)
    for r in range(12):
        nz = np.argwhere(eta[r] != 0)
        assert len(nz) == 1 and eta[r][tuple(nz[0])] == 1
        t, z, y, x, s, c = nz[0]
        assert (t, x, y, z) == src and 3 * s + c == r
