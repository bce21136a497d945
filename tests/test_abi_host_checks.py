"""Argument checks of the C ABI that run on the host before any CUDA call,
exercised without a GPU: they return the documented status and enqueue
nothing.  Pointers handed to the checks below are only tested for NULL;
no device memory exists or is touched."""
import ctypes

import pytest

from paper_2509_18261_gb300 import pmp
from paper_2509_18261_gb300 import synthetic as syn

OK, ARG, THIN, WORKSPACE, CUDA = 0, 1, 2, 6, 7
FAKE = 0x1000  # non-NULL addresses that nothing dereferences on the host
FAKE_BUF = 0x40000000  # far from FAKE: a state at FAKE and a buffer here do not overlap


@pytest.fixture(scope="module")
def lib():
    from paper_2509_18261_gb300 import build

    L = ctypes.CDLL(build.build())
    L.pmp_create.restype = ctypes.c_int32
    L.pmp_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(pmp._Params), ctypes.c_void_p]
    L.pmp_deposit_noalloc.restype = ctypes.c_int32
    L.pmp_deposit_noalloc.argtypes = [ctypes.POINTER(pmp._Params), ctypes.POINTER(pmp._Mesh),
                                      ctypes.POINTER(pmp._Particles), ctypes.c_void_p, ctypes.POINTER(pmp._Mesh),
                                      ctypes.c_void_p]
    return L


def _create(lib, params):
    out = ctypes.c_void_p(0xdead)
    code = lib.pmp_create(ctypes.byref(out), ctypes.byref(params), None)
    return code, out.value


@pytest.mark.parametrize("kind,field,value", [
    ("feedback", "kind", 9), ("feedback", "r_K", 0.5), ("feedback", "r_K", float("nan")), ("feedback", "r_K", 7.0),
    ("feedback", "subsample", 0), ("feedback", "subsample", 9), ("feedback", "gamma", 1.0),
    ("feedback", "A_sf", 0.0), ("feedback", "A_p", -1.0), ("feedback", "mu_H", 0.0), ("feedback", "eps_K", -0.1),
    ("feedback", "RM_ej", 5.0),
    ("sink", "G", 0.0), ("sink", "dt", -1.0), ("sink", "J", 0.0), ("sink", "cap", 0.0), ("sink", "cap", 1.5),
    ("sink", "rho_min", -1e-6), ("sink", "lambda_bh", float("inf")),
])
def test_create_rejects_bad_parameters_before_any_device_work(lib, kind, field, value):
    p = pmp._params_struct(syn.feedback_params() if kind == "feedback" else syn.sink_params())
    setattr(p, field, value)
    code, out = _create(lib, p)
    assert code == ARG and out is None


def test_create_without_a_device_reports_a_cuda_error(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present: pmp_create succeeds")
    code, out = _create(lib, pmp._params_struct(syn.feedback_params()))
    assert code == CUDA and out is None


def _mesh(n, ng, data=FAKE):
    px = [v + 2 * ng for v in n]
    return pmp._Mesh(n=(ctypes.c_int32 * 3)(*n), ng=ng, periodic=(ctypes.c_int32 * 3)(1, 1, 1), reserved=0,
                     dx=1.0, field_stride=px[0] * px[1] * px[2], data=data)


def _parts(count):
    return pmp._Particles(count=count, x=FAKE, y=FAKE, z=FAKE, m=FAKE, px=FAKE, py=FAKE, pz=FAKE, e=FAKE)


def _noalloc(lib, params, state, parts, buffer, gathered=FAKE):
    return lib.pmp_deposit_noalloc(ctypes.byref(params), ctypes.byref(state), ctypes.byref(parts), gathered,
                                   ctypes.byref(buffer), None)


def _buf(n=(32, 32, 32), ng=4, data=FAKE_BUF):
    return _mesh(n, ng, data)


def test_noalloc_checks_its_arguments_on_the_host(lib):
    fb = pmp._params_struct(syn.feedback_params())
    m = _mesh((32, 32, 32), 4)
    # sinks are not offered
    assert _noalloc(lib, pmp._params_struct(syn.sink_params()), m, _parts(10), _buf()) == ARG
    # no gathered rows for a non-empty set
    assert _noalloc(lib, fb, m, _parts(10), _buf(), gathered=None) == ARG
    # state and buffer of different boxes
    assert _noalloc(lib, fb, m, _parts(10), _buf((32, 32, 16))) == ARG
    # a buffer ghost layer thinner than ceil(r_K)
    assert _noalloc(lib, fb, m, _parts(10), _buf(ng=1)) == THIN
    # NULL mesh data
    assert _noalloc(lib, fb, _mesh((32, 32, 32), 4, data=None), _parts(10), _buf()) == ARG


def test_noalloc_rejects_a_state_that_overlaps_the_buffer(lib):
    fb = pmp._params_struct(syn.feedback_params())
    m = _mesh((32, 32, 32), 4)
    assert _noalloc(lib, fb, m, _parts(10), _buf(data=FAKE)) == ARG  # the same array
    assert _noalloc(lib, fb, m, _parts(10), _buf(data=FAKE + 8 * 1000)) == ARG  # inside the state's fields
    inside = _mesh((32, 32, 32), 4, data=FAKE_BUF + 8 * 64000 * 4)  # state inside the buffer's last field
    assert _noalloc(lib, fb, inside, _parts(10), _buf()) == ARG
    # a state starting further into the buffer's last field, and a buffer
    # starting inside the state's last field: each shares cells with the other
    inside = _mesh((32, 32, 32), 4, data=FAKE_BUF + 8 * (64000 * 4 + 100))
    assert _noalloc(lib, fb, inside, _parts(10), _buf()) == ARG
    assert _noalloc(lib, fb, m, _parts(10), _buf(data=FAKE + 8 * (64000 * 4 + 63999))) == ARG
    # right after the state's last cell: no shared cell, so the call gets as
    # far as its scratch limit (a count beyond it keeps it from enqueueing)
    assert _noalloc(lib, fb, m, _parts(10_000_000), _buf(data=FAKE + 8 * 64000 * 5)) == WORKSPACE


@pytest.mark.parametrize("what", ["misaligned state", "misaligned buffer", "periodic 2", "dx inf", "dx nan",
                                  "negative ng", "field stride one cell short", "no cells along an axis"])
def test_noalloc_checks_its_meshes_as_the_context_calls_do(lib, what):
    fb = pmp._params_struct(syn.feedback_params())
    m, b = _mesh((32, 32, 32), 4), _buf()
    if what == "misaligned state":
        m.data = FAKE + 4
    elif what == "misaligned buffer":
        b.data = FAKE_BUF + 4
    elif what == "periodic 2":
        m.periodic[1] = 2
        b.periodic[1] = 2
    elif what == "dx inf":
        m.dx = b.dx = float("inf")
    elif what == "dx nan":
        m.dx = b.dx = float("nan")
    elif what == "field stride one cell short":
        b.field_stride = 40 * 40 * 40 - 1
    elif what == "no cells along an axis":
        m.n[0] = b.n[0] = 0
    else:
        m.ng = -1
    assert _noalloc(lib, fb, m, _parts(10), b) == ARG


@pytest.mark.parametrize("field,value", [("A_p", float("nan")), ("eps_K", float("nan")), ("RM_ej", float("nan")),
                                         ("RM_st", float("nan")), ("gamma", float("inf")), ("A_sf", float("inf")),
                                         ("mu_H", float("inf")), ("r_K", 0.5), ("subsample", 0)])
def test_noalloc_checks_parameters_as_pmp_create_does(lib, field, value):
    fb = pmp._params_struct(syn.feedback_params())
    setattr(fb, field, value)
    assert _noalloc(lib, fb, _mesh((32, 32, 32), 4), _parts(10), _buf()) == ARG


def test_noalloc_rejects_counts_beyond_its_fixed_scratch(lib):
    # 64 MiB at 28 + 8 * 81 bytes per particle (r_K = 2): about 99,000 particles
    fb = pmp._params_struct(syn.feedback_params())
    m, b = _mesh((64, 64, 64), 4), _buf((64, 64, 64))
    assert _noalloc(lib, fb, m, _parts(120_000), b) == WORKSPACE
    assert _noalloc(lib, fb, m, _parts(10_000_000), b) == WORKSPACE
