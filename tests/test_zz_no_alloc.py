"""The per-replica energy entry point that allocates nothing on the device
(for callers that cannot allocate while reading energies, e.g. when another
framework's caching allocator holds the GPU's memory, or in monitoring code
where a cudaFree would synchronise the device), against the existing result
(ctbop_get energy) on consecutive calls. Kept in
its own file, collected last, so it runs both alone in a fresh process (the
first call then does the one-time symbol lookup) and after every other
test."""
import numpy as np
import pytest

from paper_1802_07871_gb300 import ctbop
from paper_1802_07871_gb300 import structures as st

pytestmark = pytest.mark.gpu
P1 = st.load_params("p1")


def _dimer(d, box=20.0):
    x = np.array([[5.0, 5.0, 5.0], [5.0 + d, 5.0, 5.0]])
    return st.Structure("dimer", x, np.array([0, 1], np.int32), np.full(3, box), np.array([False] * 3))


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_noalloc_energy_matches_get_on_consecutive_calls(prec):
    structs = [st.stepped_slab_small(8, 4, 6), st.bulk_3c_512(), _dimer(1.9)]
    sysm = ctbop.System(P1, precision=prec)
    sysm.load_replicas(structs)
    v = np.concatenate([st.maxwell_boltzmann(s.types, 1500.0, seed=7 + k, frozen=s.frozen)
                        for k, s in enumerate(structs)])
    sysm.set_velocities(v)
    sysm.compute()
    for _ in range(2):
        ref = sysm.get("energy")
        a = sysm.energy_noalloc()
        b = sysm.energy_noalloc()                   # second call on the same state
        np.testing.assert_allclose(a, ref, rtol=1e-12, atol=1e-9)
        np.testing.assert_allclose(b, ref, rtol=1e-12, atol=1e-9)
        sysm.step(3, 0.5)                           # new positions, charges, energies
    sysm.close()


def test_noalloc_energy_rejects_too_many_replicas():
    structs = [_dimer(1.9 + 0.001 * k) for k in range(65)]
    sysm = ctbop.System(P1, precision="mixed")
    sysm.load_replicas(structs)
    sysm.compute()
    with pytest.raises(ctbop.CtbopError, match="INVALID_ARG"):
        sysm.energy_noalloc()
    sysm.close()


def test_noalloc_energy_needs_an_evaluation():
    sysm = ctbop.System(P1, precision="mixed")
    sysm.load(_dimer(1.9))
    with pytest.raises(ctbop.CtbopError, match="STATE"):
        sysm.energy_noalloc()
    sysm.close()
