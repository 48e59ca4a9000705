"""All-gather callbacks for a j partition over several GPUs (kirin_set_j_partition).

The j-split of Sect. 3.2 lifted across GPUs: every rank keeps the whole
particle set, sums its own part of the j tiles, and the library adds every
part's seven partial sums per i in part order after the callback below has
gathered them.  These classes only move the gathered bytes (argument
marshalling); the force sums and their addition run in libkirin's kernels.

* :class:`TorchAllGather`: one rank per process over ``torch.distributed``
  (NCCL for CUDA device buffers; gloo for host buffers).
* :class:`LocalAllGather`: several contexts in one process, one host thread
  each (for example one per GPU of a node); the parts meet at a host
  barrier and copy each other's buffers device to device, so no kernel ever
  waits for another.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np


class _CudaBuffer:
    """A CUDA array interface over n float64 at a device address (for torch.as_tensor)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 2}


def device_view(ptr: int, n: int, device):
    """float64 CUDA tensor of n elements sharing the device memory at ptr."""
    import torch
    return torch.as_tensor(_CudaBuffer(ptr, n), device=device)


def host_view(ptr: int, n: int):
    """float64 CPU tensor of n elements sharing the host memory at ptr."""
    import torch
    return torch.from_numpy(np.ctypeslib.as_array((ctypes.c_double * int(n)).from_address(int(ptr))))


class TorchAllGather:
    """recv[r * count : (r + 1) * count] = send of rank r, over a torch.distributed group.

    device: the CUDA device of the context's buffers (NCCL), or "cpu" for host buffers (gloo; used by
    the CPU tests of the partition logic).  On CUDA the collective is ordered on the context's stream:
    it starts after the work already enqueued there and the library's next work waits for it."""

    def __init__(self, group=None, device="cuda"):
        import torch
        self.group = group
        self.device = torch.device(device)

    def __call__(self, send: int, recv: int, count: int, stream) -> int:
        import torch
        import torch.distributed as dist
        world = dist.get_world_size(self.group)
        if self.device.type == "cuda":
            snd = device_view(send, count, self.device)
            rcv = device_view(recv, count * world, self.device)
            ext = torch.cuda.ExternalStream(int(stream or 0), device=self.device)
            with torch.cuda.stream(ext):
                dist.all_gather_into_tensor(rcv, snd, group=self.group)
        else:
            snd = host_view(send, count)
            rcv = host_view(recv, count * world)
            dist.all_gather(list(rcv.view(world, count).unbind(0)), snd, group=self.group)
        return 0


class LocalAllGather:
    """The parts of a j partition as host threads of one process, one context each.

    ``for_part(r)`` is the callback of part r's context; each thread drives its own context and every
    force call of every part must be made (the parts meet at a barrier inside it).  devices[r] is the
    CUDA device of part r's context."""

    def __init__(self, devices, timeout: float = 60.0):
        self.devices = list(devices)
        self.n = len(self.devices)
        self.barrier = threading.Barrier(self.n, timeout=timeout)
        self.sends = [None] * self.n

    def for_part(self, part: int):
        return lambda send, recv, count, stream: self._call(part, send, recv, count, stream)

    def _call(self, part, send, recv, count, stream) -> int:
        import torch
        dev = torch.device("cuda", self.devices[part])
        ext = torch.cuda.ExternalStream(int(stream or 0), device=dev)
        ext.synchronize()  # this part's partial sums are complete
        self.sends[part] = (send, count)
        self.barrier.wait()
        with torch.cuda.stream(ext):
            rcv = device_view(recv, count * self.n, dev)
            for r in range(self.n):
                ptr, cnt = self.sends[r]
                if cnt != count:
                    raise RuntimeError(f"part {r} gathers {cnt} values, part {part} {count}")
                rcv[r * count:(r + 1) * count].copy_(device_view(ptr, count, torch.device("cuda", self.devices[r])))
        ext.synchronize()
        self.barrier.wait()  # no part refills its send buffer before every part has copied it
        return 0
