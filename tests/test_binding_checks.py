"""The Python binding refuses buffers the kernels must never see -- host tensors, tensors of the wrong
size, type or layout -- before it calls the library, so these checks run without a GPU."""
import numpy as np
import pytest
import torch

from paper_1605_05712_gb300 import api, lattice_plan, synth

S = [synth.iso_voigt(1.0, 1.0), synth.iso_voigt(10.0, 10.0)]


def test_host_tensors_are_refused():
    P = lattice_plan([[16, 4], [0, 8]])
    ph = torch.zeros(P.m, dtype=torch.uint8)                      # a host tensor
    E = np.eye(3)[:2]
    for call in (lambda: api.basic_scheme_solve(P, ph, S, (5.5, 5.5), E),
                 lambda: api.basic_scheme_solve_async(P, ph, S, (5.5, 5.5), E),
                 lambda: api.basic_scheme_solve_noalloc(P, ph, S, (5.5, 5.5), E),
                 lambda: api.basic_scheme_solve_batch(P, [ph], [S], [(5.5, 5.5)], E[:1]),
                 lambda: api.basic_scheme_solve_multi([dict(plan=P, phase=ph, stiffness=S, C0=(5.5, 5.5), E=E)]),
                 lambda: api.basic_scheme_solve_field(P, torch.zeros(21, P.m, dtype=torch.float64), (5.5, 5.5), E),
                 lambda: api.lattice_fft(P, torch.zeros(2, P.m, dtype=torch.complex128)),
                 lambda: api.gather(torch.zeros(P.m), torch.zeros(4, dtype=torch.int32))):
        with pytest.raises(TypeError):
            call()


def test_buffer_checks():
    dev = torch.device("cpu")
    good = torch.empty(2, 3, 10, dtype=torch.float64)
    assert api._on_device(good, dev) is False                     # CUDA tensors only
    with pytest.raises(TypeError):
        api._strain_buffer(good, "eps_out", 60, dev)
    with pytest.raises(TypeError):
        api._workspace(torch.empty(8, dtype=torch.uint8), 8, dev)
    # a warm start is copied into the solve's buffer: size and type are checked, layout is not
    eps = torch.empty(2, 3, 10, dtype=torch.float64)
    e0 = torch.randn(3, 2, 10, dtype=torch.float64).transpose(0, 1)
    api._fill_start(eps, e0, 60)
    assert torch.equal(eps, e0)
    for bad in (torch.randn(1, 3, 10, dtype=torch.float64), torch.randn(2, 3, 10, dtype=torch.float32)):
        with pytest.raises(TypeError):
            api._fill_start(eps, bad, 60)


def test_start_filter_refuses_host_tensors():
    from paper_1605_05712_gb300.warmstart import start_filter
    a = torch.zeros(2, 3, 5, dtype=torch.float64)
    with pytest.raises(TypeError):
        start_filter(a, a, a, 0.5)
