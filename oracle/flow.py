"""Exact integer max-flow and maximal minimum cut (test infrastructure).

Dinic's algorithm (Dinic 1970) on integer capacities held as Python ints.
The paper leaves the max-flow algorithm open (it cites Orlin's O(nm) bound);
any exact algorithm gives the same flow value and the same maximal source side
of a minimum cut, which is the set of nodes that cannot reach the sink in the
final residual graph (the cut that maximises |A|, proof of Lemma 9).

Pins (tests/test_oracle_stages.py): flow value equals the capacity of the
reported cut; value and cut side equal brute force over all s-t cuts on small
random networks.
"""
from __future__ import annotations

from collections import deque


class FlowNetwork:
    def __init__(self, num_nodes: int):
        self.n = num_nodes
        self.head = [[] for _ in range(num_nodes)]
        self.to = []
        self.cap = []

    def add_edge(self, a: int, b: int, c: int) -> int:
        """Arc a->b with capacity c (and its residual twin).  Returns the arc id."""
        self.head[a].append(len(self.to))
        self.to.append(b)
        self.cap.append(int(c))
        self.head[b].append(len(self.to))
        self.to.append(a)
        self.cap.append(0)
        return len(self.to) - 2

    def max_flow(self, s: int, t: int) -> int:
        total = 0
        while True:
            level = [-1] * self.n
            level[s] = 0
            dq = deque([s])
            while dq:
                x = dq.popleft()
                for e in self.head[x]:
                    if self.cap[e] > 0 and level[self.to[e]] < 0:
                        level[self.to[e]] = level[x] + 1
                        dq.append(self.to[e])
            if level[t] < 0:
                return total
            it = [0] * self.n
            while True:
                f = self._augment(s, t, level, it)
                if f == 0:
                    break
                total += f

    def _augment(self, s, t, level, it):
        # iterative DFS along level-increasing arcs with current-arc pointers
        path = []
        x = s
        while True:
            if x == t:
                f = min(self.cap[e] for e in path)
                for e in path:
                    self.cap[e] -= f
                    self.cap[e ^ 1] += f
                return f
            advanced = False
            while it[x] < len(self.head[x]):
                e = self.head[x][it[x]]
                y = self.to[e]
                if self.cap[e] > 0 and level[y] == level[x] + 1:
                    path.append(e)
                    x = y
                    advanced = True
                    break
                it[x] += 1
            if not advanced:
                if not path:
                    return 0
                level[x] = -1          # dead end
                e = path.pop()
                x = self.to[e ^ 1]
                it[x] += 1

    def reaches_sink(self, t: int):
        """Nodes with a residual path to t."""
        seen = [False] * self.n
        seen[t] = True
        dq = deque([t])
        while dq:
            y = dq.popleft()
            for e in self.head[y]:
                # arc e goes y -> x; its twin e^1 goes x -> y with residual cap
                x = self.to[e]
                if not seen[x] and self.cap[e ^ 1] > 0:
                    seen[x] = True
                    dq.append(x)
        return seen

    def maximal_source_side(self, t: int):
        seen = self.reaches_sink(t)
        return [i for i in range(self.n) if not seen[i]]
