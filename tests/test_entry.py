"""The entry points' host side: smoke() builds the oracle from the library's
parameters; every oracle parameter must map to a library one (checked here
without a GPU, so a renamed or added parameter cannot break the GPU smoke run)."""


def test_smoke_builds_the_oracle_from_library_parameters(orc):
    import __graft_entry__ as entry
    from paper_2002_00250_gb300 import fos
    d = fos.default_params().as_dict()
    kw = entry._oracle_pbas_params(d)
    assert set(kw) == set(orc.PBAS_DEFAULTS)
    orc.PBAS(3, 2, **kw)
    orc.GMM(3, 2, **{k: d[k] for k in orc.GMM_DEFAULTS})
