"""Host-side encodings the tensor-core GEMM issues, against the field layout
of the tcgen05 shared-memory matrix descriptor and the kind::f16 instruction
descriptor (PTX ISA): every field placed independently here."""
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1903_12359_gb300 import build
    build.build()
    from paper_1903_12359_gb300 import api
    return api.load()


def field(v, lo, width):
    return (v >> lo) & ((1 << width) - 1)


@pytest.mark.parametrize("saddr,lbo,sbo", [(0x0, 128, 1024), (0x1230, 128, 2048), (0x3FFF0, 256, 16 * 128)])
def test_smem_descriptor_fields(lib, saddr, lbo, sbo):
    d = lib.pgcp_selftest_umma_desc(saddr, lbo, sbo)
    assert field(d, 0, 14) == (saddr >> 4) & 0x3FFF        # start address >> 4
    assert field(d, 14, 2) == 0
    assert field(d, 16, 14) == lbo >> 4                     # leading byte offset >> 4
    assert field(d, 30, 2) == 0
    assert field(d, 32, 14) == sbo >> 4                     # stride byte offset >> 4
    assert field(d, 46, 3) == 0b001                         # fixed version bits
    assert field(d, 49, 3) == 0                             # base offset
    assert field(d, 52, 1) == 0                             # relative leading offset
    assert field(d, 53, 8) == 0
    assert field(d, 61, 3) == 0                             # no swizzle


@pytest.mark.parametrize("m,n", [(128, 16), (128, 64), (128, 128)])
def test_instruction_descriptor_fields(lib, m, n):
    d = lib.pgcp_selftest_umma_idesc(m, n)
    assert field(d, 0, 4) == 0           # dense, no saturate
    assert field(d, 4, 2) == 1           # D = F32
    assert field(d, 6, 1) == 0
    assert field(d, 7, 3) == 1           # A = BF16
    assert field(d, 10, 3) == 1          # B = BF16
    assert field(d, 13, 2) == 0          # no negation
    assert field(d, 15, 2) == 0          # A, B K-major
    assert field(d, 17, 6) == n >> 3
    assert field(d, 23, 1) == 0
    assert field(d, 24, 5) == m >> 4
    assert field(d, 29, 3) == 0
