"""Where page-locked host buffers sit relative to the GPU.

Host-pointer calls move every base of a batch over the CPU-GPU link (the
paper's Sec. I setting: read pairs staged from host memory into the
processing units' memory and the results read back).  On a machine with
several host NUMA nodes the link rate depends on which node holds the
page-locked buffers: a buffer on the GPU's own node goes straight over the
link, one on another node crosses the inter-socket fabric first.  Page-locked
memory is placed on the node of the CPU the allocating thread runs on, so a
process that is scheduled on the far node allocates far buffers and keeps
them for its whole life.

``bind_to_gpu(device)`` restricts the calling thread (and the threads it
starts afterwards) to the CPUs local to the GPU, when the process may run
there; call it before allocating page-locked buffers.  ``placement(addresses)``
reports which nodes hold a set of buffers, from ``/proc/self/numa_maps``.
Everything here is best effort: on a machine without the sysfs files or
without several nodes it reports what it could read and binds nothing.
"""

from __future__ import annotations

import bisect
import os
import re
import subprocess


def _read(path: str) -> str | None:
    try:
        with open(path) as f:
            return f.read().strip()
    except OSError:
        return None


def parse_cpulist(text: str | None) -> set[int]:
    """CPUs of a sysfs list such as '0-3,8,10-11'."""
    cpus: set[int] = set()
    for part in (text or "").split(","):
        part = part.strip()
        if not part:
            continue
        if "-" in part:
            a, b = part.split("-", 1)
            cpus.update(range(int(a), int(b) + 1))
        else:
            cpus.add(int(part))
    return cpus


def format_cpulist(cpus) -> str:
    """The inverse of parse_cpulist: sorted ranges."""
    out, run = [], []
    for c in sorted(cpus):
        if run and c == run[-1] + 1:
            run.append(c)
            continue
        if run:
            out.append(str(run[0]) if len(run) == 1 else "%d-%d" % (run[0], run[-1]))
        run = [c]
    if run:
        out.append(str(run[0]) if len(run) == 1 else "%d-%d" % (run[0], run[-1]))
    return ",".join(out)


def pci_address(device: int = 0) -> str | None:
    """The GPU's PCI address in sysfs form (dddd:bb:dd.f), from the CUDA
    device properties, else from nvidia-smi matched by UUID."""
    import torch

    props = torch.cuda.get_device_properties(device)
    dom, bus, dev = (getattr(props, k, None) for k in ("pci_domain_id", "pci_bus_id", "pci_device_id"))
    if None not in (dom, bus, dev):
        return "%04x:%02x:%02x.0" % (dom, bus, dev)
    uuid = str(getattr(props, "uuid", "")).lower()
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=uuid,pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=30).stdout
    except (OSError, subprocess.SubprocessError):
        return None
    for line in out.splitlines():
        parts = [p.strip() for p in line.split(",")]
        if len(parts) == 2 and uuid and uuid in parts[0].lower():
            m = re.match(r"([0-9a-fA-F]+):([0-9a-fA-F]+):([0-9a-fA-F]+)\.([0-7])", parts[1])
            if m:
                return "%04x:%s:%s.%s" % (int(m.group(1), 16), m.group(2).lower(), m.group(3).lower(), m.group(4))
    return None


def cpu_node(cpu: int, sysfs: str = "/sys/devices/system/cpu") -> int | None:
    """The NUMA node of a CPU (its nodeN link in sysfs)."""
    try:
        for name in os.listdir(os.path.join(sysfs, "cpu%d" % cpu)):
            if name.startswith("node") and name[4:].isdigit():
                return int(name[4:])
    except OSError:
        pass
    return None


def current_cpu() -> int | None:
    """The CPU the calling thread runs on (field 39 of /proc/thread-self/stat)."""
    stat = _read("/proc/thread-self/stat") or _read("/proc/self/stat")
    if not stat:
        return None
    fields = stat[stat.rfind(")") + 2:].split()  # fields 3, 4, ... after the command name
    try:
        return int(fields[36])
    except (IndexError, ValueError):
        return None


def gpu_locality(device: int = 0, sysfs_pci: str = "/sys/bus/pci/devices") -> dict:
    """The GPU's host NUMA node and its local CPUs, as sysfs lists them."""
    return locality_of(pci_address(device), sysfs_pci)


def locality_of(addr: str | None, sysfs_pci: str = "/sys/bus/pci/devices") -> dict:
    """Host NUMA node and local CPUs of the PCI device at addr."""
    info = {"pci": addr, "node": None, "local_cpus": None}
    if addr:
        node = _read(os.path.join(sysfs_pci, addr, "numa_node"))
        info["node"] = int(node) if node not in (None, "") and int(node) >= 0 else None
        info["local_cpus"] = _read(os.path.join(sysfs_pci, addr, "local_cpulist"))
    return info


def bind_to_gpu(device: int = 0) -> dict:
    """Restrict the calling thread to the GPU's local CPUs that the process
    may use.  Returns what was found and done: the GPU's node and local CPUs,
    the CPUs allowed before, whether the set changed, and the node of the
    CPU the thread runs on afterwards."""
    loc = gpu_locality(device)
    allowed = os.sched_getaffinity(0)
    local = parse_cpulist(loc["local_cpus"]) & allowed
    bound = bool(local) and local != allowed
    if bound:
        os.sched_setaffinity(0, local)
    cpu = current_cpu()
    return {"gpu_node": loc["node"], "gpu_local_cpus": loc["local_cpus"], "allowed_cpus": format_cpulist(allowed),
            "bound": bound, "thread_node": cpu_node(cpu) if cpu is not None else None}


def parse_numa_maps(text: str) -> list[tuple[int, dict[int, int]]]:
    """(start address, {node: pages}) of each mapping in a numa_maps text."""
    out = []
    for line in text.splitlines():
        parts = line.split()
        if not parts:
            continue
        try:
            start = int(parts[0], 16)
        except ValueError:
            continue
        nodes = {}
        for p in parts[1:]:
            m = re.fullmatch(r"N(\d+)=(\d+)", p)
            if m:
                nodes[int(m.group(1))] = int(m.group(2))
        out.append((start, nodes))
    out.sort()
    return out


def placement(addresses, numa_maps: str | None = None) -> dict[int, int]:
    """Pages per node of the mappings that hold the given addresses (each
    mapping counted once), from /proc/self/numa_maps."""
    maps = parse_numa_maps(numa_maps if numa_maps is not None else (_read("/proc/self/numa_maps") or ""))
    starts = [s for s, _ in maps]
    seen, total = set(), {}
    for a in addresses:
        i = bisect.bisect_right(starts, int(a)) - 1
        if i < 0 or i in seen:
            continue
        seen.add(i)
        for node, pages in maps[i][1].items():
            total[node] = total.get(node, 0) + pages
    return total
