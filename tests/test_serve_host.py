"""Host-side scheduling rules of the serving loop, checked on the CPU with
stand-ins for its streams and batches (no device work):

* a new batch takes a stream that no batch in flight uses, and falls back
  to round robin only when every stream is busy;
* a completed batch's pinned copy of the device error word decides whether
  the word is taken: a clear word costs no call, a set bit takes the word
  and marks the batch and every batch still in flight."""
from types import SimpleNamespace

import torch

import paper_cs_0004013_gb300 as rs
from paper_cs_0004013_gb300 import serve
from paper_cs_0004013_gb300.serve import SortServer


def _server(streams, in_flight_streams, next_batch=0):
    return SimpleNamespace(streams=streams, next_batch=next_batch,
                           in_flight=[SimpleNamespace(stream=s) for s in in_flight_streams])


def test_stream_prefers_one_no_batch_uses():
    a, b, c = object(), object(), object()
    assert SortServer._stream(_server([a, b, c], [a], next_batch=0)) is b
    assert SortServer._stream(_server([a, b, c], [b, c], next_batch=1)) is a
    assert SortServer._stream(_server([a, b, c], [], next_batch=2)) is c


def test_stream_round_robin_when_all_are_busy():
    a, b = object(), object()
    assert SortServer._stream(_server([a, b], [a, b], next_batch=3)) is b
    assert SortServer._stream(_server([a, b], [b, a], next_batch=4)) is a


def _fake_server(in_flight_ids):
    return SimpleNamespace(err_words=[], err_stream=None, suspect={},
                           in_flight=[SimpleNamespace(id=i) for i in in_flight_ids])


def test_clear_word_takes_nothing(monkeypatch):
    calls = []
    monkeypatch.setattr(serve, "rs_check_device_error", lambda stream=None: calls.append(stream))
    srv = _fake_server([5, 6])
    b = SimpleNamespace(id=4, err_word=torch.zeros(1, dtype=torch.int32))
    SortServer._check_errors(srv, b)
    assert calls == [] and srv.suspect == {}
    assert b.err_word is None and len(srv.err_words) == 1  # the pinned word goes back to the pool


def test_set_bit_takes_the_word_and_marks_batches_in_flight(monkeypatch):
    def take(stream=None):
        raise rs.RsError(4, "a bounded device-side wait gave up (error word 0x1)")
    monkeypatch.setattr(serve, "rs_check_device_error", take)
    srv = _fake_server([7, 8])
    b = SimpleNamespace(id=6, err_word=torch.ones(1, dtype=torch.int32))
    SortServer._check_errors(srv, b)
    assert set(srv.suspect) == {6, 7, 8}
    assert all("RS_ERR_TIMEOUT" in m for m in srv.suspect.values())


def test_set_bit_already_taken_still_marks(monkeypatch):
    """Another check took the word first (the take finds it clear): the
    batch whose copy saw the bit is still marked, with the bit it saw."""
    monkeypatch.setattr(serve, "rs_check_device_error", lambda stream=None: None)
    srv = _fake_server([])
    b = SimpleNamespace(id=9, err_word=torch.full((1,), 2, dtype=torch.int32))
    SortServer._check_errors(srv, b)
    assert set(srv.suspect) == {9} and "0x2" in srv.suspect[9] and "RS_ERR_CUDA" in srv.suspect[9]
