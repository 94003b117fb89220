"""Memory-based admission of the novel-view server (host logic, no GPU): a batch takes requests
from the head of the queue while they fit the memory budget next to what is in flight; a request
larger than the whole budget is served alone once nothing else is in flight; requests that do not
fit wait."""
from paper_2402_17427_gb300.serving import admit


def test_requests_that_fit_are_batched_up_to_the_limit():
    assert admit([10, 10, 10], 0, False, budget=100, max_batch=8) == 3
    assert admit([10] * 12, 0, False, budget=1000, max_batch=8) == 8


def test_the_budget_cuts_the_batch_and_the_rest_queue():
    assert admit([40, 40, 40], 0, False, budget=100, max_batch=8) == 2
    assert admit([40, 40, 40], 30, True, budget=100, max_batch=8) == 1
    assert admit([40, 40], 70, True, budget=100, max_batch=8) == 0      # waits for a completion


def test_an_oversized_request_runs_alone_only_when_nothing_is_in_flight():
    assert admit([500, 10], 0, False, budget=100, max_batch=8) == 1
    assert admit([500, 10], 20, True, budget=100, max_batch=8) == 0
    assert admit([500], 0, False, budget=100, max_batch=8) == 1


def test_an_empty_queue_admits_nothing():
    assert admit([], 0, False, budget=100, max_batch=8) == 0
