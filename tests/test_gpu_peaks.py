"""The throughput probes run and return rates in the range a GB300 can
reach (loose bounds: they only catch a probe that measures nothing or
overflows its timing)."""
import pytest

from paper_2311_04517_gb300 import hpclust as H

pytestmark = pytest.mark.gpu

BOUNDS = {H.HPC_PROBE_FFMA: (5e12, 1e14), H.HPC_PROBE_FFMA2: (5e12, 2e14),
          H.HPC_PROBE_DFMA: (1e10, 1e14), H.HPC_PROBE_FMIN: (1e12, 1e14),
          H.HPC_PROBE_L2_READ: (1e12, 1e14), H.HPC_PROBE_HBM_READ: (1e12, 2e13)}


@pytest.mark.parametrize("kind", sorted(BOUNDS))
def test_probe_rates(kind):
    rate, ms = H.hpc_peak_probe(kind)
    lo, hi = BOUNDS[kind]
    assert lo < rate < hi, (H.PROBES[kind], rate)
    assert ms > 0


def test_probe_rejects_unknown_kind():
    with pytest.raises(H.HPCError):
        H.hpc_peak_probe(17)
