"""The roofline probes run and report sane rates: the shared-memory atomic unit
(R_atom) and distributed shared memory across cluster ranks."""
import pytest

from paper_1111_3297_gb300 import sieve as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_probes_report_rates():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_3297_gb300 import build
    build.build_library()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    r_atom = S.sieve_probe_smem_atomics(0)
    assert 1e11 < r_atom < 32 * nsm * 4e9  # at most one 32-lane wavefront per SM-clock at 4 GHz
    for c in (2, 4, 8):
        own, ctas = S.sieve_probe_dsmem_atomics(0, c, peer=False)
        peer, ctas2 = S.sieve_probe_dsmem_atomics(0, c, peer=True)
        assert 0 < ctas == ctas2 <= nsm and ctas % c == 0
        assert 0 < peer and 0 < own < 1.5 * r_atom
    with pytest.raises(S.SieveError):
        S.sieve_probe_dsmem_atomics(0, 3)
