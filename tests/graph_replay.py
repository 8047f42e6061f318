"""Run a step the way bench.py times it (test helper): two warm-up calls on a
side stream, the step captured into a CUDA graph, one replay.  Returns the
graph's output tensors and the graph (keep it alive while they are used)."""


def replay(step, warmup=2):
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(warmup):
            step()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        out = step()
    g.replay()
    torch.cuda.synchronize()
    return out, g
