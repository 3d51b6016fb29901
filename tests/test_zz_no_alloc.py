"""The per-replica energy entry point that allocates nothing on the device
(for callers that cannot allocate while reading energies, e.g. when another
framework's caching allocator holds the GPU's memory, or in monitoring code
where a cudaFree would synchronise the device), against the existing result
(ctbop_get energy) on consecutive calls; free device memory unchanged over
many calls; and the same check in a fresh child process, where the system
created there is the first to look up the scratch array. Kept in its own
file, collected last, so it also runs after every other test."""
import os
import subprocess
import sys

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


def test_noalloc_energy_leaves_free_device_memory_unchanged():
    torch = pytest.importorskip("torch")
    structs = [st.stepped_slab_small(8, 4, 6), _dimer(1.9)]
    sysm = ctbop.System(P1, precision="mixed")
    sysm.load_replicas(structs)
    sysm.compute()
    ref = sysm.get("energy")
    sysm.energy_noalloc()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(50):
        np.testing.assert_allclose(sysm.energy_noalloc(), ref, rtol=1e-12, atol=1e-9)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    sysm.close()
    assert free1 == free0


def test_noalloc_energy_in_a_fresh_process():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import numpy as np\n"
        "from paper_1802_07871_gb300 import ctbop, structures as st\n"
        "s = st.bulk_3c_512()\n"
        "y = ctbop.System(st.load_params('p1'), precision='mixed')\n"
        "y.load(s)\n"
        "y.compute()\n"
        "a, b, ref = y.energy_noalloc(), y.energy_noalloc(), y.get('energy')\n"
        "assert np.allclose(a, ref, rtol=1e-12, atol=1e-9) and np.allclose(b, ref, rtol=1e-12, atol=1e-9)\n"
        "print('NOALLOC_OK')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "NOALLOC_OK" in r.stdout, r.stdout + r.stderr
