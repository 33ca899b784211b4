"""The paper's convergence study (Sec. 5.2.2) run through the CUDA library
gives the same E and BC as the same study run through the oracle."""
import pytest

from paper_2508_13986_gb300.convergence import temporal_study
from test_convergence import oracle_run, rotation


@pytest.mark.gpu
def test_temporal_study_through_the_library_matches_the_oracle():
    import __graft_entry__ as ge
    from paper_2508_13986_gb300.convergence import gpu_runner

    ge.build()
    w = rotation()
    gpu = temporal_study(w, eps=(0.8, 0.4), eps_ref=0.1, run=gpu_runner())
    orc = temporal_study(w, eps=(0.8, 0.4), eps_ref=0.1, run=oracle_run)
    for a, b in zip(gpu, orc):
        assert a.E == pytest.approx(b.E, abs=1e-10) and a.BC == pytest.approx(b.BC, abs=1e-10)


@pytest.mark.gpu
def test_temporal_series_through_the_library_matches_the_oracle():
    """Read-outs at intermediate times through the library equal the oracle's,
    so E(t) and BC(t) agree at every sample."""
    import __graft_entry__ as ge
    from paper_2508_13986_gb300.convergence import gpu_runner, temporal_series

    ge.build()
    times = [0.0, 0.1, 0.25, 0.4]
    gpu = temporal_series(rotation(), eps=(0.8,), eps_ref=0.2, times=times, run=gpu_runner())
    orc = temporal_series(rotation(), eps=(0.8,), eps_ref=0.2, times=times, run=oracle_run)
    for a, b in zip(gpu[0.8], orc[0.8]):
        assert a.t == b.t
        assert a.E == pytest.approx(b.E, abs=1e-10) and a.BC == pytest.approx(b.BC, abs=1e-10)
