"""Host logic of the Python binding on CPU, against a stand-in for the C
library: the server binding holds each request's input tensor and basis
until the request has completed (wait, drain or close), since the library
reads the input asynchronously; and tensor arguments are checked before any
call reaches the library."""
import ctypes as C

import pytest

torch = pytest.importorskip("torch")
import paper_2507_07788_gb300 as cq  # noqa: E402


class FakeLib:
    """Records server calls; tickets count up from 1."""

    def __init__(self):
        self.next = 0
        self.calls = []

    def cqr_server_create(self, opts, out):
        out._obj.value = 1234
        return cq.OK

    def _submit(self, kind, ticket):
        self.next += 1
        ticket._obj.value = self.next
        self.calls.append((kind, self.next))
        return cq.OK

    def cqr_server_submit_factor(self, h, b, n, ptr, lda, opts, ticket):
        return self._submit("factor", ticket)

    def cqr_server_submit_append(self, h, b, p, ptr, lda, ticket):
        return self._submit("append", ticket)

    def cqr_server_wait(self, h, ticket, out):
        self.calls.append(("wait", ticket))
        return cq.OK

    def cqr_server_drain(self, h):
        self.calls.append(("drain", None))
        return cq.OK

    def cqr_server_destroy(self, h):
        self.calls.append(("destroy", None))
        return cq.OK


class FakeBasis:
    _h = C.c_void_p(5678)


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib()
    monkeypatch.setattr(cq, "_lib", f)
    return f


def colmajor_cpu(m, n):
    return torch.zeros((n, m), dtype=torch.float64).t()


def test_server_holds_inputs_until_completion(fake):
    srv = cq.Server()
    b = FakeBasis()
    A, B, Cin = colmajor_cpu(10, 3), colmajor_cpu(10, 2), colmajor_cpu(10, 1)
    t1 = srv.submit_factor(b, A)
    t2 = srv.submit_append(b, B)
    t3 = srv.submit_append(b, Cin)
    assert set(srv._held) == {t1, t2, t3}
    assert srv._held[t2][0] is B and srv._held[t2][1] is b
    srv.wait(t2)
    assert set(srv._held) == {t1, t3}
    srv.drain()
    assert srv._held == {}
    t4 = srv.submit_append(b, B)
    assert set(srv._held) == {t4}
    srv.close()
    assert srv._held == {} and ("destroy", None) in fake.calls


def test_tensor_arguments_are_checked_first(fake):
    srv = cq.Server()
    b = FakeBasis()
    with pytest.raises(TypeError):
        srv.submit_append(b, torch.zeros((10, 2), dtype=torch.float32))
    with pytest.raises(ValueError):
        srv.submit_append(b, torch.zeros((10, 2), dtype=torch.float64))  # row-major
    assert not any(k in ("factor", "append") for k, _ in fake.calls)
    assert srv._held == {}
    srv.close()
